// dev_linalg.cuh -- small dense linear algebra for one thread group.
//
// A "group" is NT threads (one warp, or several warps joined by a named
// barrier) that cooperates on one matrix operation.  Operands live in shared
// memory (or global memory for read-only operands), row-major with an
// explicit leading dimension; every size is a compile-time constant so the
// loops unroll.  Each operation ends with a group barrier unless told not to,
// so its result may be read by any thread of the group afterwards.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace pdl {

__host__ __device__ constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ constexpr int round4(int a) { return (a + 3) & ~3; }

// ------------------------------------------------ asynchronous copies
// Global -> shared copies that bypass registers (cp.async): a group issues
// every copy of a tile, then waits once, so all loads of the tile are in
// flight together.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(NPEND) : "memory"); }

// Copy COUNT floats of one stage (global offset base + gs * COUNT) into shared
// memory with the group's threads.  16-byte copies when every address of the
// tile is 16-byte aligned by construction (COUNT a multiple of 4 and a 16-byte
// aligned shared destination and global base), 4-byte copies otherwise.
// A destination outside shared memory (kernels whose work areas live in a
// global workspace) is filled with plain vector loads and stores instead.
template <int COUNT, int NT, bool VEC>
__device__ __forceinline__ void stage_copy(int t, float* dst, const float* src)
{
    if (!__isShared(dst)) {
        if constexpr (VEC && COUNT % 4 == 0) {
            for (int e = t; e < COUNT / 4; e += NT)
                reinterpret_cast<float4*>(dst)[e] = __ldg(reinterpret_cast<const float4*>(src) + e);
        } else {
            for (int e = t; e < COUNT; e += NT) dst[e] = src[e];
        }
        return;
    }
    if constexpr (VEC && COUNT % 4 == 0) {
        for (int e = t; e < COUNT / 4; e += NT) cp_async16(dst + 4 * e, src + 4 * e);
    } else {
        for (int e = t; e < COUNT; e += NT) cp_async4(dst + e, src + e);
    }
}

// MUFU reciprocal and reciprocal square root (about 1 ulp); used on the
// sequential critical path of the factorisations, whose results are FP32 and
// are corrected by the refinement step where the residual matters.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int NT>
struct Grp {
    int t;    // rank inside the group
    int bar;  // named barrier id (groups wider than one warp)
    float* tb = nullptr;  // the group's shared-memory tile buffer (TileBuf), or none
    float* fb = nullptr;  // the group's shared-memory factor buffer, or none
    int fbn = 0;          // its size in floats
    struct TcCtx* tc = nullptr;  // tensor-core context of the CTA (TMEM, barrier), or none
    unsigned mask = 0xffffffffu; // lanes of a group narrower than a warp (NT = 16: one half)
    __device__ __forceinline__ void sync() const {
        if constexpr (NT == 32) {
            __syncwarp();
        } else if constexpr (NT == 16) {
            __syncwarp(mask);
        } else {
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(NT) : "memory");
        }
    }
};

// Register tile (RT x CT) for an R x C result spread over NT threads: the
// smallest tile whose tile count fits in NT, ties broken by fewer operand
// loads (RT + CT); tiles are capped at 4 x 4 (larger results loop).
template <int R, int C, int NT>
struct TilePick {
    __host__ __device__ static constexpr int pick() {
        for (int area = 1; area <= 16; ++area) {
            int best = -1, best_cost = 1 << 30;
            for (int rt = 1; rt <= 4; ++rt) {
                if (area % rt) continue;
                int ct = area / rt;
                if (ct > 4) continue;
                if (cdiv(R, rt) * cdiv(C, ct) > NT) continue;
                if (rt + ct < best_cost) { best_cost = rt + ct; best = rt * 8 + ct; }
            }
            if (best >= 0) return best;
        }
        return 4 * 8 + 4;
    }
    static constexpr int RT = pick() / 8;
    static constexpr int CT = pick() % 8;
};

// Opt-in dynamic shared memory of one CTA on sm_103a.
constexpr size_t kSmemCta = 227 * 1024;

// ------------------------------------------------ tensor-core products
// A CTA that takes products through the tensor cores owns columns of tensor
// memory (one 128-lane fp32 accumulator of up to TMEM_TILE columns per
// 128-row output tile) and an mbarrier on which each batch of MMAs signals
// completion.
constexpr int TMEM_TILE = 256;

struct TcCtx {
    uint64_t mbar;     // completion barrier of the issued MMAs
    uint32_t tmem;     // TMEM address of the accumulators
    uint32_t ncols;    // columns allocated (TMEM_TILE per 128-row tile)
    uint32_t phase;    // parity the next wait expects
    int failed;        // a wait ran out (the products written as NaN)
    int skip_issue;    // test switch: issue neither the MMAs nor their commit,
                       // so that the bounded wait runs out with nothing in flight
};

// Limits of the wait for a batch of MMAs (which completes in microseconds):
// the wait itself, and the second wait for MMAs still in flight after it ran
// out, before the staging buffers and the tensor memory are reused or freed.
constexpr uint64_t kTcWaitNs = 500000000ull;
constexpr uint64_t kTcDrainNs = 100000000ull;

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Poll phase `phase` of an mbarrier until it completes or limit_ns pass (also
// capped in polls); returns whether it completed.  The clock is first read
// after 64 polls, so that a wait that completes at once costs no timer read.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t phase, uint64_t limit_ns)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0; it < (1u << 28); ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"((uint32_t)__cvta_generic_to_shared(mbar)), "r"(phase) : "memory");
        if (done) return true;
        if ((it & 63) == 63) {
            const uint64_t now = globaltimer_ns();
            if (it == 63) t0 = now;
            else if (now - t0 > limit_ns) return false;
        }
    }
    return false;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ------------------------------------------------ bulk copies (TMA engine)
// One-dimensional bulk copy from global to this CTA's shared memory on the
// tensor memory accelerator, completing as transaction bytes on an mbarrier.
// dst and src must be 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(mbar)) : "memory");
}

// mbarrier with `count` arrivals per phase (call from one thread, then make
// the initialisation visible with mbar_init_fence and a CTA barrier).
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// The calling thread's arrival on the current phase, announcing `bytes` of
// bulk copies that complete on it.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(mbar)), "r"(bytes) : "memory");
}
// Orders this thread's earlier shared-memory accesses (generic proxy) before
// later bulk copies into the same locations (async proxy).
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Allocate ncols columns (TMEM_TILE per 128-row tile of the largest
// product; a power of two, at most 512) and set up the barrier (all threads
// of the CTA).
__device__ __forceinline__ void tc_setup(TcCtx* c, uint32_t ncols, bool skip_issue = false)
{
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&c->tmem)), "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&c->mbar)));
        c->ncols = ncols;
        c->phase = 0;
        c->failed = 0;
        c->skip_issue = skip_issue ? 1 : 0;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Release the accumulator (all threads of the CTA, after its last product).
__device__ __forceinline__ void tc_teardown(TcCtx* c)
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(c->tmem), "r"(c->ncols));
}

// Shared-memory matrix descriptor of a K-major tile without swizzle: core
// matrices of 8 rows x 16 bytes, 128 bytes apart along K and 256 bytes
// apart along the rows (descriptor version 1).
__device__ __forceinline__ uint64_t tc_sdesc(const void* p)
{
    const uint64_t a = smem_u32(p);
    return ((a & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) | (1ull << 46);
}

// Offset (floats) of element (r, k), k < 8, in such a tile.
__device__ __forceinline__ int tc_koff(int r, int k) { return (r >> 3) * 64 + (k >> 2) * 32 + (r & 7) * 4 + (k & 3); }

__device__ __forceinline__ float tf32_round(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// 128-row output tiles of an R-row product, and the floats of staging the
// product needs (high and low TF32 parts of a K-chunk of 32 of both operands).
__host__ __device__ constexpr int tc_mtiles(int R) { return (R + 127) / 128; }
__host__ __device__ constexpr int tc_stage_floats(int R, int C)
{
    return 2 * 4 * 128 * 8 * tc_mtiles(R) + 2 * 4 * C * 8;
}
// TMEM columns a CTA whose products have up to R rows allocates.
__host__ __device__ constexpr int tc_cols(int R) { return tc_mtiles(R) > 1 ? 512 : TMEM_TILE; }

// Tile buffer of a wide group's shared-memory tiled product: a K-chunk of
// op(A) (BK x BM, k-major) and of op(B) (BK x BN), rows padded to LDT.
struct TileBuf {
    static constexpr int BM = 64, BN = 64, BK = 32, LDT = 68;
    static constexpr int FLOATS = 2 * BK * LDT;
};

// out[R][C] = D + sgn * op(A) op(B) for a group of NT = 128 or 256 threads
// through its tile buffer: 64 x 64 output tiles; per K-chunk of 32 the group
// copies op(A) and op(B) into shared memory (coalesced along the operands'
// contiguous index, zero-filled beyond the edges), then every thread
// accumulates a 4 x TC register tile from float4 reads.  Operands may live in
// global or shared memory; out may alias D but not A or B.
template <int R, int C, int K, bool TA, bool TB, int NT>
__device__ void mm_tiled(const Grp<NT>& g, float* out, int ldo, const float* A, int lda,
                         const float* B, int ldb, const float* D, int ldd, float sgn)
{
    static_assert(NT == 128 || NT == 256, "tiled product groups");
    constexpr int BM = TileBuf::BM, BN = TileBuf::BN, BK = TileBuf::BK, LDT = TileBuf::LDT;
    constexpr int TC = BM * BN / (NT * 4);   // 4 (NT = 256) or 8 (NT = 128) columns
    constexpr int CG = BN / TC;              // column groups
    float* As = g.tb;
    float* Bs = g.tb + BK * LDT;
    const int tx = g.t % CG, ty = g.t / CG;
    for (int r0 = 0; r0 < R; r0 += BM) {
        for (int c0 = 0; c0 < C; c0 += BN) {
            float acc[4][TC];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < TC; ++j) acc[i][j] = 0.f;
            // K-chunks: every load of a chunk is issued before its first
            // shared store (through generic pointers the compiler cannot
            // order them otherwise), then the chunk is multiplied
            constexpr int NL = BM * BK / NT;
            for (int k0 = 0; k0 < K; k0 += BK) {
                {
                    float va[NL];
#pragma unroll
                    for (int q = 0; q < NL; ++q) {
                        // As[l][r] = op(A)(r0 + r, k0 + l)
                        const int e = g.t + q * NT;
                        const int r = TA ? e % BM : e / BK, l = TA ? e / BM : e % BK;
                        const int gr = r0 + r, gl = k0 + l;
                        va[q] = ((R % BM == 0 || gr < R) && (K % BK == 0 || gl < K))
                                    ? (TA ? A[(size_t)gl * lda + gr] : A[(size_t)gr * lda + gl]) : 0.f;
                    }
#pragma unroll
                    for (int q = 0; q < NL; ++q) {
                        const int e = g.t + q * NT;
                        const int r = TA ? e % BM : e / BK, l = TA ? e / BM : e % BK;
                        As[l * LDT + r] = va[q];
                    }
                }
                {
                    float vb[NL];
#pragma unroll
                    for (int q = 0; q < NL; ++q) {
                        // Bs[l][c] = op(B)(k0 + l, c0 + c)
                        const int e = g.t + q * NT;
                        const int c = TB ? e / BK : e % BN, l = TB ? e % BK : e / BN;
                        const int gc = c0 + c, gl = k0 + l;
                        vb[q] = ((C % BN == 0 || gc < C) && (K % BK == 0 || gl < K))
                                    ? (TB ? B[(size_t)gc * ldb + gl] : B[(size_t)gl * ldb + gc]) : 0.f;
                    }
#pragma unroll
                    for (int q = 0; q < NL; ++q) {
                        const int e = g.t + q * NT;
                        const int c = TB ? e / BK : e % BN, l = TB ? e % BK : e / BN;
                        Bs[l * LDT + c] = vb[q];
                    }
                }
                g.sync();
#pragma unroll 8
                for (int l = 0; l < BK; ++l) {
                    const float4 a = *reinterpret_cast<const float4*>(As + l * LDT + ty * 4);
                    float b[TC];
#pragma unroll
                    for (int q = 0; q < TC / 4; ++q) {
                        const float4 bq = *reinterpret_cast<const float4*>(Bs + l * LDT + tx * TC + 4 * q);
                        b[4 * q] = bq.x; b[4 * q + 1] = bq.y; b[4 * q + 2] = bq.z; b[4 * q + 3] = bq.w;
                    }
                    const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < TC; ++j) acc[i][j] = fmaf(av[i], b[j], acc[i][j]);
                }
                g.sync();
            }
            // addends first, then the stores (out may alias D)
            if (D) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = r0 + ty * 4 + i;
#pragma unroll
                    for (int j = 0; j < TC; ++j) {
                        const int c = c0 + tx * TC + j;
                        const bool in = (R % BM == 0 || r < R) && (C % BN == 0 || c < C);
                        acc[i][j] = sgn * acc[i][j] + (in ? D[(size_t)r * ldd + c] : 0.f);
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < TC; ++j) acc[i][j] *= sgn;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = r0 + ty * 4 + i;
                if (R % BM != 0 && r >= R) continue;
#pragma unroll
                for (int j = 0; j < TC; ++j) {
                    const int c = c0 + tx * TC + j;
                    if (C % BN != 0 && c >= C) continue;
                    out[(size_t)r * ldo + c] = acc[i][j];
                }
            }
        }
    }
}

// out[R][C] = D + sgn * op(A) op(B)   (D == nullptr: no addend)
// op(A)(r,l) = TA ? A[l*lda + r] : A[r*lda + l];  op(B)(l,c) likewise.
// out must not alias A or B; it may alias D.
// out[R][C] = D + sgn * op(A) op(B) on the tensor cores, for a group of 256
// threads that is its whole CTA.  Each 128-row output tile accumulates in its
// own TMEM columns (tile i at column TMEM_TILE i).  Per K-chunk of 32 the
// group copies op(A) and op(B) asynchronously straight into K-major
// positions of the factor buffer (no register round trip, all copies in
// flight together), splits every value in place into TF32 high and low parts
// (x = hi + lo), and one thread issues, per tile and K-step of 8, the products
// lo(A) hi(B), hi(A) lo(B) and hi(A) hi(B) (kind::tf32, M = 128, N = C), which
// recover FP32 accuracy (lo(A) lo(B) is below FP32 rounding).  The
// accumulators are read back by 32x32b loads (warp w: lanes 32 (w mod 4) ..,
// its warpgroup's 16-column slices).  Every wait is bounded; if one runs out
// the product is written as NaN and the CTA's context marked failed.
template <int R, int C, int K, bool TA, bool TB, int NT>
__device__ void mm_tc(const Grp<NT>& g, float* out, int ldo, const float* A, int lda,
                      const float* B, int ldb, const float* D, int ldd, float sgn)
{
    static_assert(NT == 256 && C % 32 == 0 && C <= TMEM_TILE && K % 8 == 0, "tensor-core shapes");
    constexpr int KC = 32, MT = tc_mtiles(R), AT = 128 * 8, BT = C * 8;
    constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(C >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
    TcCtx* cx = g.tc;
    float* Ahi = g.fb;                  // [MT][4][AT]
    float* Alo = Ahi + MT * 4 * AT;
    float* Bhi = Alo + MT * 4 * AT;     // [4][BT]
    float* Blo = Bhi + 4 * BT;
    const int t = g.t, warp = t >> 5, lane = t & 31;
    uint32_t phase = cx->phase;
    bool failed = cx->failed != 0;
    const uint32_t tmem = cx->tmem;
    for (int k0 = 0; k0 < K; k0 += KC) {
        const int kn = (K - k0) < KC ? (K - k0) : KC;   // multiple of 8
        // op(A) rows 0..MT*128-1 (zero beyond R) and op(B), K-major; operands
        // in shared memory are copied by plain loads and stores
        const bool ash = __isShared(A), bsh = __isShared(B);
        for (int e = t; e < MT * 128 * KC; e += NT) {
            const int r = TA ? e % (MT * 128) : e / KC, k = TA ? e / (MT * 128) : e % KC;
            float* d = Ahi + (r >> 7) * 4 * AT + (k >> 3) * AT + tc_koff(r & 127, k & 7);
            if (r < R && k < kn) {
                const float* src = TA ? A + (size_t)(k0 + k) * lda + r : A + (size_t)r * lda + k0 + k;
                if (ash) *d = *src;
                else cp_async4(d, src);
            } else {
                *d = 0.f;
            }
        }
        for (int e = t; e < C * KC; e += NT) {
            const int c = TB ? e / KC : e % C, k = TB ? e % KC : e / C;
            float* d = Bhi + (k >> 3) * BT + tc_koff(c, k & 7);
            if (k < kn) {
                const float* src = TB ? B + (size_t)c * ldb + k0 + k : B + (size_t)(k0 + k) * ldb + c;
                if (bsh) *d = *src;
                else cp_async4(d, src);
            } else {
                *d = 0.f;
            }
        }
        cp_async_commit();
        cp_async_wait_all();
        g.sync();
        // split in place: hi stays, lo goes to the parallel buffer
        for (int e = t; e < MT * 4 * AT; e += NT) {
            const float x = Ahi[e], h = tf32_round(x);
            Ahi[e] = h;
            Alo[e] = tf32_round(x - h);
        }
        for (int e = t; e < 4 * BT; e += NT) {
            const float x = Bhi[e], h = tf32_round(x);
            Bhi[e] = h;
            Blo[e] = tf32_round(x - h);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        g.sync();
        if (t == 0 && !failed && !cx->skip_issue) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int mt = 0; mt < MT; ++mt) {
                const uint32_t d = tmem + (uint32_t)(mt * TMEM_TILE);
                for (int s = 0; s < kn / 8; ++s) {
                    const float* ah = Ahi + mt * 4 * AT + s * AT;
                    const float* al = Alo + mt * 4 * AT + s * AT;
                    const uint32_t first = (k0 == 0 && s == 0) ? 0u : 1u;
                    tc_mma(d, tc_sdesc(al), tc_sdesc(Bhi + s * BT), IDESC, first);
                    tc_mma(d, tc_sdesc(ah), tc_sdesc(Blo + s * BT), IDESC, 1u);
                    tc_mma(d, tc_sdesc(ah), tc_sdesc(Bhi + s * BT), IDESC, 1u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&cx->mbar)) : "memory");
        }
        if (!failed) {
            const bool done = mbar_wait_bounded(&cx->mbar, phase, kTcWaitNs);
            // one verdict for the whole CTA (the group is the CTA), so that
            // the TMEM loads below run on all warps or on none; the barrier
            // also orders the next chunk's staging after every thread's wait
            failed = __syncthreads_or(done ? 0 : 1) != 0;
            phase ^= 1;
            if (failed) {
                // MMAs possibly still in flight get a second bounded wait
                // before their operands and accumulators are given up
                if (!done) mbar_wait_bounded(&cx->mbar, phase ^ 1, kTcDrainNs);
                g.sync();
            }
        } else {
            g.sync();
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (failed) break;   // uniform: no further chunk is staged or issued
    }
    // read the accumulators back: out = D + sgn * acc.  A lane holds one row
    // of a warp's 32 x 16 slice; the slice goes through the (now idle)
    // staging area so that the addend loads and the stores run along rows.
    float* tb = g.fb + warp * 32 * 17;
    for (int mt = 0; mt < MT; ++mt) {
        const int rbase = mt * 128 + 32 * (warp & 3);
        for (int c0 = (warp >> 2) * 16; c0 < C; c0 += 32) {
            uint32_t v[16];
            if (!failed) {
                const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(mt * TMEM_TILE + c0);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                               "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                               "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                             : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = 0x7fc00000u;   // NaN
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) tb[lane * 17 + j] = __uint_as_float(v[j]);
            __syncwarp();
            // lane (h, c): column c0 + c of rows rbase + h, + 2, ...
            const int c = lane & 15, h = lane >> 4;
            float o[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int rr = h + 2 * i, gr = rbase + rr;
                o[i] = sgn * tb[rr * 17 + c] + ((D && gr < R) ? D[(size_t)gr * ldd + c0 + c] : 0.f);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int gr = rbase + h + 2 * i;
                if (gr < R) out[(size_t)gr * ldo + c0 + c] = o[i];
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    g.sync();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (t == 0) {
        cx->phase = phase;
        cx->failed = failed ? 1 : 0;
    }
}

template <int R, int C, int K, bool TA, bool TB, int NT, bool SYNC = true>
__device__ __forceinline__ void mm(const Grp<NT>& g, float* out, int ldo,
                                   const float* A, int lda, const float* B, int ldb,
                                   const float* D = nullptr, int ldd = 0, float sgn = 1.f)
{
    // a CTA-wide group with a tensor-core context takes large products there
    if constexpr (NT == 256 && R >= 64 && C >= 64 && C % 32 == 0 && C <= TMEM_TILE && K >= 32 &&
                  K % 8 == 0) {
        if (g.tc && g.fb && g.fbn >= tc_stage_floats(R, C) && g.tc->ncols >= (uint32_t)tc_cols(R)) {
            mm_tc<R, C, K, TA, TB, NT>(g, out, ldo, A, lda, B, ldb, D, ldd, sgn);
            g.sync();
            return;
        }
    }
    // wide groups with a tile buffer take large products through shared memory
    if constexpr ((NT == 128 || NT == 256) && R >= 48 && C >= 48 && K >= 32) {
        if (g.tb) {
            mm_tiled<R, C, K, TA, TB, NT>(g, out, ldo, A, lda, B, ldb, D, ldd, sgn);
            if constexpr (SYNC) g.sync();
            return;
        }
    }
    constexpr int RT = TilePick<R, C, NT>::RT, CT = TilePick<R, C, NT>::CT;
    constexpr int TR = cdiv(R, RT), TC = cdiv(C, CT), NTILE = TR * TC;
    for (int tile = g.t; tile < NTILE; tile += NT) {
        const int r0 = (tile / TC) * RT, c0 = (tile % TC) * CT;
        float acc[RT][CT];
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
            for (int j = 0; j < CT; ++j) acc[i][j] = 0.f;
#pragma unroll(K <= 24 ? K : 8)
        for (int l = 0; l < K; ++l) {
            float a[RT], b[CT];
#pragma unroll
            for (int i = 0; i < RT; ++i) {
                const int r = (R % RT == 0) ? r0 + i : min(r0 + i, R - 1);
                a[i] = TA ? A[l * lda + r] : A[r * lda + l];
            }
#pragma unroll
            for (int j = 0; j < CT; ++j) {
                const int c = (C % CT == 0) ? c0 + j : min(c0 + j, C - 1);
                b[j] = TB ? B[c * ldb + l] : B[l * ldb + c];
            }
#pragma unroll
            for (int i = 0; i < RT; ++i)
#pragma unroll
                for (int j = 0; j < CT; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        // addends first, then the stores (out may alias D)
#pragma unroll
        for (int i = 0; i < RT; ++i) {
            const int r = r0 + i;
#pragma unroll
            for (int j = 0; j < CT; ++j) {
                const int c = c0 + j;
                const bool in = (R % RT == 0 || r < R) && (C % CT == 0 || c < C);
                acc[i][j] = sgn * acc[i][j] + ((D && in) ? D[r * ldd + c] : 0.f);
            }
        }
#pragma unroll
        for (int i = 0; i < RT; ++i) {
            const int r = r0 + i;
            if (R % RT != 0 && r >= R) continue;
#pragma unroll
            for (int j = 0; j < CT; ++j) {
                const int c = c0 + j;
                if (C % CT != 0 && c >= C) continue;
                out[r * ldo + c] = acc[i][j];
            }
        }
    }
    if constexpr (SYNC) g.sync();
}

// y[R] = d + sgn * op(A) x   (matrix-vector, a one-column mm)
template <int R, int K, bool TA, int NT, bool SYNC = true>
__device__ __forceinline__ void mv(const Grp<NT>& g, float* y, const float* A, int lda,
                                   const float* x, const float* d = nullptr, float sgn = 1.f)
{
    mm<R, 1, K, TA, false, NT, SYNC>(g, y, 1, A, lda, x, 1, d, 1, sgn);
}

// dst[R][C] = src (optionally transposed source)
template <int R, int C, bool TS, int NT, bool SYNC = true>
__device__ __forceinline__ void copy(const Grp<NT>& g, float* dst, int ldd, const float* src, int lds)
{
    for (int e = g.t; e < R * C; e += NT) {
        const int r = e / C, c = e % C;
        dst[r * ldd + c] = TS ? src[c * lds + r] : src[r * lds + c];
    }
    if constexpr (SYNC) g.sync();
}

template <int R, int C, int NT, bool SYNC = true>
__device__ __forceinline__ void fill(const Grp<NT>& g, float* dst, int ldd, float v, float diag = 0.f)
{
    for (int e = g.t; e < R * C; e += NT) {
        const int r = e / C, c = e % C;
        dst[r * ldd + c] = (r == c) ? diag : v;
    }
    if constexpr (SYNC) g.sync();
}

// M <- (M + M^T) / 2 for an N x N matrix (removes rounding asymmetry).
template <int N, int NT, bool SYNC = true>
__device__ __forceinline__ void symmetrize(const Grp<NT>& g, float* M, int ld)
{
    for (int e = g.t; e < N * N; e += NT) {
        const int r = e / N, c = e % N;
        if (c > r) {
            const float v = 0.5f * (M[r * ld + c] + M[c * ld + r]);
            M[r * ld + c] = v;
            M[c * ld + r] = v;
        }
    }
    if constexpr (SYNC) g.sync();
}

// In-place Cholesky of an SPD M x M matrix (lower triangle, right-looking).
// dinv[j] receives 1 / L[j][j].  Returns false (uniformly over the group) if
// a pivot is not positive and finite; the factor is then meaningless.
template <int M, int NT>
__device__ bool chol_generic(const Grp<NT>& g, float* L, int ld, float* dinv)
{
    bool ok = true;
    for (int j = 0; j < M; ++j) {
        const float d = L[j * ld + j];
        ok = ok && (d > 0.f) && isfinite(d);
        const float s = sqrtf(fmaxf(d, 1e-30f));
        const float inv = 1.f / s;
        g.sync();
        for (int i = j + 1 + g.t; i < M; i += NT) L[i * ld + j] *= inv;
        if (g.t == 0) {
            L[j * ld + j] = s;
            dinv[j] = inv;
        }
        g.sync();
        const int rem = M - j - 1;
        for (int e = g.t; e < rem * rem; e += NT) {
            const int i = j + 1 + e / rem, k = j + 1 + e % rem;
            if (k <= i) L[i * ld + k] -= L[i * ld + j] * L[k * ld + j];
        }
        g.sync();
    }
    return ok;
}

// Solve L Y = X in place (X is M x NC); L lower triangular, dinv = 1/diag.
template <int M, int NC, int NT>
__device__ void trsm_lower_generic(const Grp<NT>& g, const float* L, int ld, const float* dinv,
                                   float* X, int ldx)
{
    for (int i = 0; i < M; ++i) {
        for (int c = g.t; c < NC; c += NT) X[i * ldx + c] *= dinv[i];
        g.sync();
        const int rows = M - i - 1;
        for (int e = g.t; e < rows * NC; e += NT) {
            const int r = i + 1 + e / NC, c = e % NC;
            X[r * ldx + c] -= L[r * ld + i] * X[i * ldx + c];
        }
        g.sync();
    }
}

// Solve L^T Y = X in place (X is M x NC).
template <int M, int NC, int NT>
__device__ void trsm_lower_t_generic(const Grp<NT>& g, const float* L, int ld, const float* dinv,
                                     float* X, int ldx)
{
    for (int i = M - 1; i >= 0; --i) {
        for (int c = g.t; c < NC; c += NT) X[i * ldx + c] *= dinv[i];
        g.sync();
        for (int e = g.t; e < i * NC; e += NT) {
            const int r = e / NC, c = e % NC;
            X[r * ldx + c] -= L[i * ld + r] * X[i * ldx + c];
        }
        g.sync();
    }
}

// Gauss-Jordan elimination with partial pivoting on the augmented matrix
// [Mx | RHS] (Mx is N x N in columns 0..N-1, NR right-hand sides after it)
// by a group of NT threads, one column per thread.  Step k exchanges rows k
// and p (the pivot row) and eliminates column k from every other row, over
// the columns right of the pivot; column k itself is read but never written
// in the step (the exchange is applied to it virtually), and the pivot row
// is not normalised, so one barrier per step suffices.  The thread that
// updates column k + 1 also finds the next pivot row and publishes the
// column as the next step's multipliers in the group's tile buffer
// (double-buffered; without one the multipliers are read from column k).
// Columns are processed in register chunks of rows.  On exit columns
// N..N+NR-1 hold Mx^{-1} RHS (each row divided by its pivot).  wsc: 2 N
// floats.  Returns false (uniformly) if a pivot is zero or not finite.
template <int N, int NR, int NT>
__device__ bool gj_solve_generic(const Grp<NT>& g, float* G, int ld, float* wsc)
{
    constexpr int W = N + NR;
    constexpr int RB = 12;
    int* prow = reinterpret_cast<int*>(wsc);   // [N] pivot rows
    float* dpiv = wsc + N;                     // [N] pivots
    float* mbuf = (g.tb && 2 * N <= TileBuf::FLOATS) ? g.tb : nullptr;
    if (mbuf)
        for (int i = g.t; i < N; i += NT) mbuf[i] = G[(size_t)i * ld];
    if (g.t == 0) {
        int bi = 0;
        float best = -1.f;
        for (int i = 0; i < N; ++i) {
            const float v = fabsf(G[(size_t)i * ld]);
            if (v > best) { best = v; bi = i; }
        }
        prow[0] = bi;
    }
    g.sync();
    bool ok = true;
    for (int k = 0; k < N; ++k) {
        const float* mc = mbuf ? mbuf + (k & 1) * N : nullptr;   // column k
        float* mnext = mbuf ? mbuf + ((k + 1) & 1) * N : nullptr;
        const int p = prow[k];
        const float dk = mc ? mc[p] : G[(size_t)p * ld + k];
        ok = ok && (fabsf(dk) > 1e-30f) && isfinite(dk);
        const float idk = 1.f / dk;
        const float mk = mc ? mc[k] : G[(size_t)k * ld + k];   // multiplier of row p after the exchange
        for (int j = k + 1 + g.t; j < W; j += NT) {
            float* col = G + j;
            const float vk = col[(size_t)p * ld], vp = col[(size_t)k * ld];
            col[(size_t)k * ld] = vk;             // pivot row
            const float rk = vk * idk;
            const bool next = (j == k + 1);
            const bool pub = mnext && next && j < N;
            float best = -1.f;
            int bi = k + 1;
            // rows in batches: every load of a batch (multipliers from the
            // staged column when present) is issued before the batch's stores
            for (int i0 = 0; i0 < N; i0 += RB) {
                float mv[RB], cv[RB];
#pragma unroll
                for (int q = 0; q < RB; ++q) {
                    const int i = i0 + q;
                    const bool in = N % RB == 0 || i < N;
                    mv[q] = in ? (mc ? mc[i] : G[(size_t)i * ld + k]) : 0.f;
                    cv[q] = in ? col[(size_t)i * ld] : 0.f;
                }
#pragma unroll
                for (int q = 0; q < RB; ++q) {
                    const int i = i0 + q;
                    if (N % RB == 0 || i < N) {
                        // the pivot row keeps vk (stored again with the same
                        // value), row p takes the exchanged row k's entry
                        const bool ik = (i == k), ip = (i == p) && !ik;
                        const float u = fmaf(-(ip ? mk : mv[q]), rk, ip ? vp : cv[q]);
                        const float v = ik ? vk : u;
                        col[(size_t)i * ld] = v;
                        if (pub) mnext[i] = v;
                        if (next && i > k && fabsf(v) > best) { best = fabsf(v); bi = i; }
                    }
                }
            }
            if (next && k + 1 < N) prow[k + 1] = bi;
        }
        if (g.t == 0) dpiv[k] = dk;
        g.sync();
    }
    for (int e = g.t; e < N * NR; e += NT) {
        const int i = e / NR, c = e - i * NR;
        G[(size_t)i * ld + N + c] *= 1.f / dpiv[i];
    }
    g.sync();
    return ok;
}

// Gauss-Jordan elimination with partial pivoting of [M | RHS] (N rows, N + NR
// columns, row-major with leading dimension ld) in FP64: the FP32 entries
// are widened once and every thread of the group holds one column in FP64
// registers for the whole elimination.  Rows are exchanged implicitly: the
// pivot row of step k is recorded (prow[k]), not moved, so no register array
// is indexed by a run-time row.  At step k the owner of column k publishes
// that column (the multipliers) and its pivot row, chosen by the largest
// magnitude among the rows not yet used, to a double-buffered FP64 area; the
// owner of column k + 1 publishes the next one right after its own update,
// so a step costs one barrier.  Every column j > k then divides its entry in
// the pivot row by the pivot and subtracts the multiples from the other rows.
// On exit the pivot row of step k holds row k of M^-1 RHS, which is written
// back (rounded to FP32) over G's columns N.. at row k.  dbuf: 2 N doubles +
// 2 N ints of shared memory (or work-area memory).  Returns false (uniformly)
// if a pivot's magnitude is below 1e-300 or not finite.
template <int N, int NR, int NT>
__device__ bool gj_solve_f64(const Grp<NT>& g, float* G, int ld, double* dbuf)
{
    constexpr int W = N + NR;
    static_assert(W <= NT, "one column per thread");
    static_assert(N <= 64, "used rows as a 64-bit mask");
    double* mcol = dbuf;                                  // [2][N] multiplier columns
    int* prow = reinterpret_cast<int*>(dbuf + 2 * N);    // [N] pivot row of step k
    int* rank = prow + N;                                 // [N] step at which row i pivots
    const int j = g.t;
    const bool mine = j < W;
    double c[N];
#pragma unroll
    for (int i = 0; i < N; ++i) c[i] = mine ? (double)G[(size_t)i * ld + j] : 0.0;
    uint64_t used = 0;
    // the owner of column k: its column as multipliers, the pivot row
    auto publish = [&](int k) {
        double* m = mcol + (k & 1) * N;
        double best = -1.0;
        int bi = 0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            m[i] = c[i];
            const double a = fabs(c[i]);
            if (!((used >> i) & 1) && a > best) { best = a; bi = i; }
        }
        prow[k] = bi;
    };
    if (j == 0) publish(0);
    g.sync();
    bool ok = true;
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
        const double* m = mcol + (k & 1) * N;
        const int p = prow[k];
        const double piv = m[p];
        ok = ok && fabs(piv) > 1e-300 && isfinite(piv);
        if (mine && j > k) {
            double vp = 0.0;
#pragma unroll
            for (int i = 0; i < N; ++i) vp = i == p ? c[i] : vp;
            const double rk = vp / piv;
#pragma unroll
            for (int i = 0; i < N; ++i) c[i] = i == p ? rk : fma(-m[i], rk, c[i]);
        }
        used |= uint64_t(1) << p;
        if (j == k + 1 && k + 1 < N) publish(k + 1);
        g.sync();
    }
    if (j == 0)
        for (int k = 0; k < N; ++k) rank[prow[k]] = k;
    g.sync();
    if (mine && j >= N) {
#pragma unroll
        for (int i = 0; i < N; ++i) G[(size_t)rank[i] * ld + j] = (float)c[i];
    }
    g.sync();
    return ok;
}

// ---------------------------------------------------------------------------
// One-warp versions: operands live in registers, one row or one column per
// lane, so the sequential steps need no index arithmetic and few barriers.

// Right-looking Cholesky, lane i holds row i (M <= 32).  Per column j: lane j
// takes the square root of its pivot, lanes below scale their entry and
// publish it, then every lane applies the rank-one update to its own row.
template <int M>
__device__ bool chol_warp(int lane, float* L, int ld, float* dinv, float* colbuf)
{
    static_assert(M <= 32, "one row per lane");
    float row[M];
#pragma unroll
    for (int k = 0; k < M; ++k) row[k] = (lane < M) ? L[lane * ld + k] : 0.f;
    bool ok = true;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        // two alternating slots: a slot is rewritten two columns later, after
        // every lane has passed the next column's first barrier
        float* cb = colbuf + (j & 1) * (M + 3);
        if (lane == j) {
            const float d = row[j];
            const float inv = rsqrt_approx(fmaxf(d, 1e-30f));
            cb[M] = (d > 0.f && isfinite(d)) ? 1.f : 0.f;
            cb[M + 1] = d * inv;
            cb[M + 2] = inv;
            dinv[j] = inv;
        }
        __syncwarp();
        ok = ok && (cb[M] != 0.f);
        const float inv = cb[M + 2];
        if (lane == j) row[j] = cb[M + 1];
        if (lane > j && lane < M) {
            row[j] *= inv;
            cb[lane] = row[j];
        }
        __syncwarp();
        if (lane > j && lane < M) {
            const float lij = row[j];
#pragma unroll
            for (int k = j + 1; k < M; ++k) row[k] -= lij * cb[k];
        }
    }
    if (lane < M) {
#pragma unroll
        for (int k = 0; k < M; ++k)
            if (k <= lane) L[lane * ld + k] = row[k];
    }
    __syncwarp();
    return ok;
}

// L Y = X with one right-hand side per lane (forward substitution in
// registers); L is read by broadcast.  NC right-hand sides, any count.
template <int M, int NC>
__device__ void trsm_lower_warp(int lane, const float* L, int ld, const float* dinv, float* X, int ldx)
{
    for (int c = lane; c < NC; c += 32) {
        float y[M];
#pragma unroll
        for (int i = 0; i < M; ++i) y[i] = X[i * ldx + c];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            float v = y[i];
#pragma unroll
            for (int l = 0; l < i; ++l) v -= L[i * ld + l] * y[l];
            y[i] = v * dinv[i];
        }
#pragma unroll
        for (int i = 0; i < M; ++i) X[i * ldx + c] = y[i];
    }
    __syncwarp();
}

// L^T Y = X, backward substitution per lane.
template <int M, int NC>
__device__ void trsm_lower_t_warp(int lane, const float* L, int ld, const float* dinv, float* X, int ldx)
{
    for (int c = lane; c < NC; c += 32) {
        float y[M];
#pragma unroll
        for (int i = 0; i < M; ++i) y[i] = X[i * ldx + c];
#pragma unroll
        for (int i = M - 1; i >= 0; --i) {
            float v = y[i];
#pragma unroll
            for (int l = i + 1; l < M; ++l) v -= L[l * ld + i] * y[l];
            y[i] = v * dinv[i];
        }
#pragma unroll
        for (int i = 0; i < M; ++i) X[i * ldx + c] = y[i];
    }
    __syncwarp();
}

// Gauss-Jordan with partial pivoting, one column of [Mx | RHS] per lane
// (two for lanes below W - 32).  Step k: lane k picks the pivot in its column,
// swaps, and publishes the column (double-buffered shared slot); every lane
// swaps the same rows of its columns, normalises the pivot row entry and
// eliminates.  Only columns right of the pivot are updated.  On exit the RHS
// columns hold Mx^{-1} RHS.  colbuf: 2 * (N + 1) floats.
template <int N, int NR>
__device__ bool gj_warp(int lane, float* G, int ld, float* colbuf)
{
    constexpr int W = N + NR;
    constexpr int NQ = (W + 31) / 32;
    static_assert(N <= 32 && NQ <= 2, "pivot columns owned by single lanes");
    float c[NQ][N];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int j = lane + 32 * q;
#pragma unroll
        for (int i = 0; i < N; ++i) c[q][i] = (j < W) ? G[i * ld + j] : 0.f;
    }
    bool ok = true;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        float* cb = colbuf + (k & 1) * (N + 1);
        if (lane == k) {
            // tree argmax of |c[0][i]| over rows k..N-1
            constexpr int R = N;   // slots; rows below k are masked out
            float v[R];
            int id[R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                v[i] = (i >= k) ? fabsf(c[0][i]) : -1.f;
                id[i] = i;
            }
#pragma unroll
            for (int w = 1; w < R; w <<= 1)
#pragma unroll
                for (int i = 0; i + w < R; i += 2 * w)
                    if (v[i + w] > v[i]) { v[i] = v[i + w]; id[i] = id[i + w]; }
            const int piv = id[0];
            float vp = c[0][k];
#pragma unroll
            for (int i = k + 1; i < N; ++i) vp = (piv == i) ? c[0][i] : vp;
#pragma unroll
            for (int i = k + 1; i < N; ++i) c[0][i] = (piv == i) ? c[0][k] : c[0][i];
            c[0][k] = vp;
#pragma unroll
            for (int i = 0; i < N; ++i) cb[i] = c[0][i];
            cb[N] = __int_as_float(piv);
        }
        __syncwarp();
        const int piv = __float_as_int(cb[N]);
        const float pk = cb[k];
        ok = ok && (fabsf(pk) > 1e-30f) && isfinite(pk);
        const float inv = rcp_approx(pk);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int j = lane + 32 * q;
            if (j <= k || j >= W) continue;
            // entry piv of the column by a binary tree of selects
            float t[N];
#pragma unroll
            for (int i = 0; i < N; ++i) t[i] = c[q][i];
#pragma unroll
            for (int w = 1; w < N; w <<= 1) {
                const bool hi = (piv & w) != 0;
#pragma unroll
                for (int i = 0; i + w < N; i += 2 * w) t[i] = hi ? t[i + w] : t[i];
            }
            const float vp = t[0];
#pragma unroll
            for (int i = k + 1; i < N; ++i) c[q][i] = (piv == i) ? c[q][k] : c[q][i];
            const float r = vp * inv;
            c[q][k] = r;
#pragma unroll
            for (int i = 0; i < N; ++i)
                if (i != k) c[q][i] -= cb[i] * r;
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int j = lane + 32 * q;
        if (j >= N && j < W) {
#pragma unroll
            for (int i = 0; i < N; ++i) G[i * ld + j] = c[q][i];
        }
    }
    __syncwarp();
    return ok;
}

// G^-1 X for an SPD M x M matrix G and NR right-hand sides X (M x NR) by
// Gauss-Jordan elimination without pivoting, one column per lane in registers:
// lane j < M holds column j of G, lane M + r holds right-hand side r.  For an
// SPD matrix the pivots are the diagonal of its L D L^T factorisation, so
// "every pivot positive and finite" is the SPD test (the one a Cholesky
// factorisation makes) and no pivot search is needed.  Step k: lane k
// publishes its column (double-buffered shared slot), every lane scales its
// row-k entry and eliminates.  Out (M x NR) receives G^-1 X; every operand is
// read before anything is written, so Out may alias X.  colbuf: 2 M floats.
// Returns false (uniformly over the warp) if a pivot is not positive and finite.
template <int M, int NR>
__device__ bool spd_solve_warp(int lane, const float* G, int ldg, const float* X, int ldx,
                               float* Out, int ldo, float* colbuf)
{
    static_assert(M + NR <= 32, "one column per lane");
    const bool isG = lane < M;
    const bool isX = lane >= M && lane < M + NR;
    float c[M];
#pragma unroll
    for (int i = 0; i < M; ++i) c[i] = isG ? G[i * ldg + lane] : (isX ? X[i * ldx + lane - M] : 0.f);
    __syncwarp();
    bool ok = true;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        // a slot is rewritten two steps later, after every lane has passed
        // the next step's barrier (and so finished reading this one)
        float* cb = colbuf + (k & 1) * M;
        if (lane == k) {
#pragma unroll
            for (int i = 0; i < M; ++i) cb[i] = c[i];
        }
        __syncwarp();
        const float pk = cb[k];
        ok = ok && (pk > 0.f) && isfinite(pk);
        const float r = c[k] * rcp_approx(pk);
        c[k] = r;
#pragma unroll
        for (int i = 0; i < M; ++i)
            if (i != k) c[i] = fmaf(-cb[i], r, c[i]);
    }
    if (isX) {
#pragma unroll
        for (int i = 0; i < M; ++i) Out[i * ldo + lane - M] = c[i];
    }
    __syncwarp();
    return ok;
}

// G^-1 X for an SPD M x M matrix G (overwritten) and NR right-hand sides X
// (overwritten by the solution) by a group of NT threads: Gauss-Jordan
// elimination without pivoting, one column of [G | X] per thread.  Step k
// subtracts G[i][k] / G[k][k] times pivot row k from every other row i over
// the columns right of the pivot and all right-hand sides; the pivot row is
// not normalised, so no entry a step reads is written in that step and one
// barrier per step suffices.  At the end every row of X is divided by its
// pivot (the pivots of an SPD matrix are the diagonal of its L D L^T
// factorisation; "all positive and finite" is the SPD test).  The thread
// that updates column k + 1 also publishes it as the next step's multipliers
// in the group's tile buffer (double-buffered), so the other threads read
// them from shared memory; without a tile buffer they read column k itself.
// Columns are processed in register chunks of rows (all loads of a chunk
// before its stores).  piv: M floats.  Returns false (uniformly over the
// group) if a pivot is not positive and finite.
template <int M, int NR, int NT>
__device__ bool spd_solve_generic(const Grp<NT>& g, float* G, int ldg, float* X, int ldx, float* piv)
{
    constexpr int W = M + NR;
    constexpr int RB = 12;
    float* mbuf = (g.tb && 2 * M <= TileBuf::FLOATS) ? g.tb : nullptr;
    if (mbuf) {
        for (int i = g.t; i < M; i += NT) mbuf[i] = G[(size_t)i * ldg];
        g.sync();
    }
    bool ok = true;
    for (int k = 0; k < M; ++k) {
        const float* mk = mbuf ? mbuf + (k & 1) * M : nullptr;
        float* mnext = mbuf ? mbuf + ((k + 1) & 1) * M : nullptr;
        const float pk = mk ? mk[k] : G[(size_t)k * ldg + k];
        ok = ok && (pk > 0.f) && isfinite(pk);
        const float ipk = 1.f / pk;
        for (int j = k + 1 + g.t; j < W; j += NT) {
            float* col = j < M ? G + j : X + (j - M);
            const int ld = j < M ? ldg : ldx;
            const float rk = col[(size_t)k * ld] * ipk;
            const bool pub = mnext && j == k + 1 && j < M;
            // rows in batches: every load of a batch (multipliers from the
            // staged column when present) is issued before the batch's stores
            for (int i0 = 0; i0 < M; i0 += RB) {
                float mv[RB], cv[RB];
#pragma unroll
                for (int q = 0; q < RB; ++q) {
                    const int i = i0 + q;
                    const bool in = M % RB == 0 || i < M;
                    mv[q] = in ? (mk ? mk[i] : G[(size_t)i * ldg + k]) : 0.f;
                    cv[q] = in ? col[(size_t)i * ld] : 0.f;
                }
#pragma unroll
                for (int q = 0; q < RB; ++q) {
                    const int i = i0 + q;
                    if (M % RB == 0 || i < M) {
                        const float v = i == k ? cv[q] : fmaf(-mv[q], rk, cv[q]);
                        col[(size_t)i * ld] = v;   // the pivot row is stored unchanged
                        if (pub) mnext[i] = v;
                    }
                }
            }
        }
        if (g.t == 0) piv[k] = pk;
        g.sync();
    }
    for (int e = g.t; e < M * NR; e += NT) {
        const int i = e / NR, c = e - i * NR;
        X[(size_t)i * ldx + c] *= 1.f / piv[i];
    }
    g.sync();
    return ok;
}

// Floats of shared memory that spd_solve_smem needs for an M x M system:
// the factor (rows padded to M + 1) and one block of SMEM_CB right-hand sides.
constexpr int SMEM_CB = 64;
__host__ __device__ constexpr int spd_smem_floats(int M) { return round4(M * (M + 1)) + M * SMEM_CB; }

// G^-1 X for an SPD M x M matrix G (global or shared, read only) and NR
// right-hand sides X (overwritten by the solution) by a group of NT threads,
// with the factorisation resident in the group's factor buffer (at least
// spd_smem_floats(M) floats): G is copied in and factored G = L L^T there
// (right-looking, column by column: the pivot row scales column j, then every
// thread updates its rows of the trailing lower triangle), and X is solved in
// blocks of SMEM_CB columns staged beside the factor (forward substitution
// L Y = X, then L^T Z = Y, one row of unknowns per step).  piv: M floats (the
// reciprocal pivots).  Returns false (uniformly) if a pivot is not positive
// and finite (G not SPD).
template <int M, int NR, int NT>
__device__ bool spd_solve_smem(const Grp<NT>& g, const float* G, int ldg, float* X, int ldx, float* piv)
{
    constexpr int LD = M + 1;   // odd row stride: threads on different rows hit different banks
    float* L = g.fb;
    float* Xs = g.fb + round4(M * LD);
    // copies into the buffer go out as asynchronous copies (all in flight at
    // once); a G already in shared memory is copied by plain loads and stores
    const bool gsh = __isShared(G);
    for (int e = g.t; e < M * M; e += NT) {
        const int i = e / M, k = e - i * M;
        if (gsh) L[i * LD + k] = G[(size_t)i * ldg + k];
        else cp_async4(L + i * LD + k, G + (size_t)i * ldg + k);
    }
    cp_async_commit();
    cp_async_wait_all();
    g.sync();
    // blocked right-looking factorisation by diagonal blocks of FB columns:
    // one warp factors the block in registers (rows per lane), one thread per
    // row below solves its panel row against the block's transpose (FB
    // unknowns in registers), then the trailing lower triangle loses
    // L21 L21^T through register tiles (thread (ty, tx): rows ty + TY q,
    // columns 4 tx .. 4 tx + 3 of each 64-column slab)
    constexpr int FB = M % 32 == 0 ? 32 : M % 16 == 0 ? 16 : M % 8 == 0 ? 8 : M % 4 == 0 ? 4
                     : M % 2 == 0 ? 2 : 1;
    // the right-hand-side area is idle during the factorisation: its first
    // word carries the "every pivot positive" flag to all threads
    float* okw = Xs;
    if (g.t == 0) okw[0] = 1.f;
    for (int jb = 0; jb < M; jb += FB) {
        const int je = jb + FB;
        if (g.t < 32) {
            // Cholesky of the FB x FB diagonal block, lane i holds row i
            const int lane = g.t;
            float row[FB];
#pragma unroll
            for (int k = 0; k < FB; ++k) row[k] = lane < FB ? L[(jb + lane) * LD + jb + k] : 0.f;
            bool okb = true;
#pragma unroll
            for (int j = 0; j < FB; ++j) {
                const float d = __shfl_sync(0xffffffffu, row[j], j);
                okb = okb && (d > 0.f) && isfinite(d);
                const float inv = rsqrtf(fmaxf(d, 1e-30f));
                if (lane == j) row[j] = d * inv;
                if (lane > j) row[j] *= inv;
                if (lane == 0) piv[jb + j] = inv;
#pragma unroll
                for (int k = j + 1; k < FB; ++k) {
                    const float lkj = __shfl_sync(0xffffffffu, row[j], k);
                    if (lane > j && k <= lane) row[k] = fmaf(-row[j], lkj, row[k]);
                }
            }
            if (lane < FB) {
#pragma unroll
                for (int k = 0; k < FB; ++k)
                    if (k <= lane) L[(jb + lane) * LD + jb + k] = row[k];
            }
            if (lane == 0 && !okb) okw[0] = 0.f;
        }
        g.sync();
        if (je < M) {
            // panel: row r below solves l_r L11^T = a_r (forward substitution)
            for (int r = je + g.t; r < M; r += NT) {
                float a[FB];
#pragma unroll
                for (int k = 0; k < FB; ++k) a[k] = L[r * LD + jb + k];
#pragma unroll
                for (int k = 0; k < FB; ++k) {
#pragma unroll
                    for (int l = 0; l < k; ++l) a[k] = fmaf(-a[l], L[(jb + k) * LD + jb + l], a[k]);
                    a[k] *= piv[jb + k];
                }
#pragma unroll
                for (int k = 0; k < FB; ++k) L[r * LD + jb + k] = a[k];
            }
            g.sync();
            // trailing update of the lower triangle of rows/columns je..M-1
            constexpr int TXC = 16, TYR = NT / TXC, QT = (M + TYR - 1) / TYR;
            const int tx = g.t % TXC, ty = g.t / TXC;
            for (int c0 = je; c0 < M; c0 += 4 * TXC) {
                const int cb = c0 + 4 * tx;   // this thread's first column
                float acc[QT][4];
#pragma unroll
                for (int q = 0; q < QT; ++q)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[q][c] = 0.f;
                for (int k = jb; k < je; ++k) {
                    float lc[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) lc[c] = cb + c < M ? L[(cb + c) * LD + k] : 0.f;
#pragma unroll
                    for (int q = 0; q < QT; ++q) {
                        const int r = c0 + ty + TYR * q;   // rows from the slab's first column down
                        const float lr = r < M ? L[r * LD + k] : 0.f;
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[q][c] = fmaf(lr, lc[c], acc[q][c]);
                    }
                }
#pragma unroll
                for (int q = 0; q < QT; ++q) {
                    const int r = c0 + ty + TYR * q;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (r < M && cb + c < M && cb + c <= r) L[r * LD + cb + c] -= acc[q][c];
                }
            }
            g.sync();
        }
    }
    const bool ok = okw[0] != 0.f;
    g.sync();   // the flag is read before the right-hand sides overwrite it
    // right-hand sides: thread (rr, cc) owns column cc of rows rr, rr + RPP, ...
    static_assert(NT % SMEM_CB == 0, "whole rows of a block per pass");
    constexpr int RPP = NT / SMEM_CB;
    const int cc = g.t % SMEM_CB, rr = g.t / SMEM_CB;
    for (int c0 = 0; c0 < NR; c0 += SMEM_CB) {
        const bool on = c0 + cc < NR;
        const bool xsh = __isShared(X);
        for (int r = rr; r < M; r += RPP)
            if (on) {
                if (xsh) Xs[r * SMEM_CB + cc] = X[(size_t)r * ldx + c0 + cc];
                else cp_async4(Xs + r * SMEM_CB + cc, X + (size_t)r * ldx + c0 + cc);
            }
        cp_async_commit();
        cp_async_wait_all();
        g.sync();
        // L Y = X by diagonal blocks of DB rows: inside a block, step i uses
        // y_i = x_i / L_ii and removes L_ri y_i from the block's later rows;
        // the block's rows are then scaled to y, and every row below loses
        // L[r][block] y[block] through a register-tiled product (thread
        // (ty, tx): four columns, rows ty, ty + 16, ...)
        // diagonal blocks of DB rows (the largest of 32, 16, ..., 1 dividing M)
        constexpr int DB = M % 32 == 0 ? 32 : M % 16 == 0 ? 16 : M % 8 == 0 ? 8 : M % 4 == 0 ? 4
                         : M % 2 == 0 ? 2 : 1;
        const int tx = g.t % 16, ty = g.t / 16;   // 16 column groups x NT / 16 row offsets
        constexpr int TY = NT / 16, QR = (M + TY - 1) / TY;
        for (int kb = 0; kb < M; kb += DB) {
            const int ke = kb + DB;
            // the block's own triangle: one thread per column, its DB unknowns
            // in registers (L read by broadcast), no barrier inside
            if (g.t < SMEM_CB) {
                float y[DB];
#pragma unroll
                for (int i = 0; i < DB; ++i) y[i] = Xs[(kb + i) * SMEM_CB + g.t];
#pragma unroll
                for (int i = 0; i < DB; ++i) {
                    y[i] *= piv[kb + i];
#pragma unroll
                    for (int r = i + 1; r < DB; ++r) y[r] = fmaf(-L[(kb + r) * LD + kb + i], y[i], y[r]);
                }
#pragma unroll
                for (int i = 0; i < DB; ++i) Xs[(kb + i) * SMEM_CB + g.t] = y[i];
            }
            g.sync();
            if (ke < M) {
                float acc[QR][4];
#pragma unroll
                for (int q = 0; q < QR; ++q)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[q][c] = 0.f;
                for (int k = kb; k < ke; ++k) {
                    const float4 y = *reinterpret_cast<const float4*>(Xs + k * SMEM_CB + 4 * tx);
#pragma unroll
                    for (int q = 0; q < QR; ++q) {
                        const int r = ke + ty + TY * q;
                        const float l = r < M ? L[r * LD + k] : 0.f;
                        acc[q][0] = fmaf(l, y.x, acc[q][0]);
                        acc[q][1] = fmaf(l, y.y, acc[q][1]);
                        acc[q][2] = fmaf(l, y.z, acc[q][2]);
                        acc[q][3] = fmaf(l, y.w, acc[q][3]);
                    }
                }
#pragma unroll
                for (int q = 0; q < QR; ++q) {
                    const int r = ke + ty + TY * q;
                    if (r < M) {
                        float4* px = reinterpret_cast<float4*>(Xs + r * SMEM_CB + 4 * tx);
                        float4 v = *px;
                        v.x -= acc[q][0]; v.y -= acc[q][1]; v.z -= acc[q][2]; v.w -= acc[q][3];
                        *px = v;
                    }
                }
                g.sync();
            }
        }
        // L^T Z = Y by the same blocks from the bottom up: rows above a block
        // lose L[block][r]^T z[block]
        for (int kb = M - DB; kb >= 0; kb -= DB) {
            const int ke = kb + DB;
            if (g.t < SMEM_CB) {
                float z[DB];
#pragma unroll
                for (int i = 0; i < DB; ++i) z[i] = Xs[(kb + i) * SMEM_CB + g.t];
#pragma unroll
                for (int i = DB - 1; i >= 0; --i) {
                    z[i] *= piv[kb + i];
#pragma unroll
                    for (int r = 0; r < i; ++r) z[r] = fmaf(-L[(kb + i) * LD + kb + r], z[i], z[r]);
                }
#pragma unroll
                for (int i = 0; i < DB; ++i) Xs[(kb + i) * SMEM_CB + g.t] = z[i];
            }
            g.sync();
            if (kb > 0) {
                float acc[QR][4];
#pragma unroll
                for (int q = 0; q < QR; ++q)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[q][c] = 0.f;
                for (int k = kb; k < ke; ++k) {
                    const float4 z = *reinterpret_cast<const float4*>(Xs + k * SMEM_CB + 4 * tx);
#pragma unroll
                    for (int q = 0; q < QR; ++q) {
                        const int r = ty + TY * q;
                        const float l = r < kb ? L[k * LD + r] : 0.f;
                        acc[q][0] = fmaf(l, z.x, acc[q][0]);
                        acc[q][1] = fmaf(l, z.y, acc[q][1]);
                        acc[q][2] = fmaf(l, z.z, acc[q][2]);
                        acc[q][3] = fmaf(l, z.w, acc[q][3]);
                    }
                }
#pragma unroll
                for (int q = 0; q < QR; ++q) {
                    const int r = ty + TY * q;
                    if (r < kb) {
                        float4* px = reinterpret_cast<float4*>(Xs + r * SMEM_CB + 4 * tx);
                        float4 v = *px;
                        v.x -= acc[q][0]; v.y -= acc[q][1]; v.z -= acc[q][2]; v.w -= acc[q][3];
                        *px = v;
                    }
                }
                g.sync();
            }
        }
        for (int r0 = rr; r0 < M; r0 += 8 * RPP) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int r = r0 + q * RPP;
                v[q] = r < M ? Xs[r * SMEM_CB + cc] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int r = r0 + q * RPP;
                if (on && r < M) X[(size_t)r * ldx + c0 + cc] = v[q];
            }
        }
        g.sync();
    }
    return ok;
}

// M^-1 X for a general M x M matrix (G, global or shared, read only; rows of
// stride ldg) and NR right-hand sides X (overwritten by the solution) by a
// group of NT threads, with the factorisation resident in the group's factor
// buffer (spd_smem_floats(M) floats, the layout of spd_solve_smem): G is
// copied in and factored P G = L U by Gauss elimination with partial pivoting
// (right-looking, unblocked: at step k warp 0 picks the row of largest
// magnitude in column k, all threads exchange the two rows whole, and every
// thread then eliminates one row below the pivot against the pivot row, read
// by broadcast), and X is solved in blocks of SMEM_CB columns staged beside
// the factor through the row permutation (forward substitution with the unit
// lower factor, then back substitution with U).  wsc: 3 M words of scratch
// (pivot rows, the row map, the reciprocal pivots).  Returns false
// (uniformly) if a pivot's magnitude is below 1e-30 or not finite.
template <int M, int NR, int NT>
__device__ bool lu_solve_smem(const Grp<NT>& g, const float* G, int ldg, float* X, int ldx, float* wsc)
{
    constexpr int LD = M + 1;   // odd row stride: threads on different rows hit different banks
    float* L = g.fb;
    float* Xs = g.fb + round4(M * LD);
    int* prow = reinterpret_cast<int*>(wsc);        // [M] pivot row of step k
    int* rmap = prow + M;                           // [M] original row at position i
    float* piv = wsc + 2 * M;                       // [M] 1 / U_kk
    const bool gsh = __isShared(G);
    for (int e = g.t; e < M * M; e += NT) {
        const int i = e / M, k = e - i * M;
        if (gsh) L[i * LD + k] = G[(size_t)i * ldg + k];
        else cp_async4(L + i * LD + k, G + (size_t)i * ldg + k);
    }
    cp_async_commit();
    cp_async_wait_all();
    // the right-hand-side area is idle during the factorisation: word 0 holds
    // the "every pivot usable" flag, word 1 the pivot row of the current step
    float* okw = Xs;
    int* pw = reinterpret_cast<int*>(Xs + 1);
    if (g.t == 0) okw[0] = 1.f;
    g.sync();
    for (int k = 0; k < M; ++k) {
        if (g.t < 32) {
            float best = -1.f;
            int bi = k;
            for (int i = k + g.t; i < M; i += 32) {
                const float a = fabsf(L[i * LD + k]);
                if (a > best) { best = a; bi = i; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (g.t == 0) {
                pw[0] = bi;
                prow[k] = bi;
                if (!(best > 1e-30f) || !isfinite(best)) okw[0] = 0.f;
            }
        }
        g.sync();
        const int p = pw[0];
        if (p != k)
            for (int c = g.t; c < M; c += NT) {
                const float a = L[k * LD + c];
                L[k * LD + c] = L[p * LD + c];
                L[p * LD + c] = a;
            }
        g.sync();
        const float ukk = L[k * LD + k];
        const float inv = 1.f / ukk;
        if (g.t == 0) piv[k] = inv;
        for (int i = k + 1 + g.t; i < M; i += NT) {
            const float l = L[i * LD + k] * inv;
            L[i * LD + k] = l;
            for (int j = k + 1; j < M; ++j) L[i * LD + j] = fmaf(-l, L[k * LD + j], L[i * LD + j]);
        }
        g.sync();
    }
    const bool ok = okw[0] != 0.f;
    if (g.t == 0) {
        for (int i = 0; i < M; ++i) rmap[i] = i;
        for (int k = 0; k < M; ++k) {
            const int p = prow[k], t = rmap[k];
            rmap[k] = rmap[p];
            rmap[p] = t;
        }
    }
    __threadfence_block();
    g.sync();   // the flag and the row map are read before the right-hand sides overwrite them
    static_assert(NT % SMEM_CB == 0, "whole rows of a block per pass");
    constexpr int RPP = NT / SMEM_CB;
    const int cc = g.t % SMEM_CB, rr = g.t / SMEM_CB;
    constexpr int DB = M % 32 == 0 ? 32 : M % 16 == 0 ? 16 : M % 8 == 0 ? 8 : M % 4 == 0 ? 4
                     : M % 2 == 0 ? 2 : 1;
    const int tx = g.t % 16, ty = g.t / 16;   // 16 column groups x NT / 16 row offsets
    constexpr int TY = NT / 16, QR = (M + TY - 1) / TY;
    for (int c0 = 0; c0 < NR; c0 += SMEM_CB) {
        const bool on = c0 + cc < NR;
        const bool xsh = __isShared(X);
        // staged through the row permutation: position r holds original row rmap[r]
        for (int r = rr; r < M; r += RPP) {
            const float* src = X + (size_t)rmap[r] * ldx + c0 + cc;
            if (!on) Xs[r * SMEM_CB + cc] = 0.f;
            else if (xsh) Xs[r * SMEM_CB + cc] = *src;
            else cp_async4(Xs + r * SMEM_CB + cc, src);
        }
        cp_async_commit();
        cp_async_wait_all();
        g.sync();
        // L Y = P X (unit lower factor) by diagonal blocks of DB rows
        for (int kb = 0; kb < M; kb += DB) {
            const int ke = kb + DB;
            if (g.t < SMEM_CB) {
                float y[DB];
#pragma unroll
                for (int i = 0; i < DB; ++i) y[i] = Xs[(kb + i) * SMEM_CB + g.t];
#pragma unroll
                for (int i = 0; i < DB; ++i)
#pragma unroll
                    for (int r = i + 1; r < DB; ++r) y[r] = fmaf(-L[(kb + r) * LD + kb + i], y[i], y[r]);
#pragma unroll
                for (int i = 0; i < DB; ++i) Xs[(kb + i) * SMEM_CB + g.t] = y[i];
            }
            g.sync();
            if (ke < M) {
                float acc[QR][4];
#pragma unroll
                for (int q = 0; q < QR; ++q)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[q][c] = 0.f;
                for (int k = kb; k < ke; ++k) {
                    const float4 y = *reinterpret_cast<const float4*>(Xs + k * SMEM_CB + 4 * tx);
#pragma unroll
                    for (int q = 0; q < QR; ++q) {
                        const int r = ke + ty + TY * q;
                        const float l = r < M ? L[r * LD + k] : 0.f;
                        acc[q][0] = fmaf(l, y.x, acc[q][0]);
                        acc[q][1] = fmaf(l, y.y, acc[q][1]);
                        acc[q][2] = fmaf(l, y.z, acc[q][2]);
                        acc[q][3] = fmaf(l, y.w, acc[q][3]);
                    }
                }
#pragma unroll
                for (int q = 0; q < QR; ++q) {
                    const int r = ke + ty + TY * q;
                    if (r < M) {
                        float4* px = reinterpret_cast<float4*>(Xs + r * SMEM_CB + 4 * tx);
                        float4 v = *px;
                        v.x -= acc[q][0]; v.y -= acc[q][1]; v.z -= acc[q][2]; v.w -= acc[q][3];
                        *px = v;
                    }
                }
                g.sync();
            }
        }
        // U Z = Y by the same blocks from the bottom up: rows above a block
        // lose U[r][block] z[block]
        for (int kb = M - DB; kb >= 0; kb -= DB) {
            const int ke = kb + DB;
            if (g.t < SMEM_CB) {
                float z[DB];
#pragma unroll
                for (int i = 0; i < DB; ++i) z[i] = Xs[(kb + i) * SMEM_CB + g.t];
#pragma unroll
                for (int i = DB - 1; i >= 0; --i) {
                    z[i] *= piv[kb + i];
#pragma unroll
                    for (int r = 0; r < i; ++r) z[r] = fmaf(-L[(kb + r) * LD + kb + i], z[i], z[r]);
                }
#pragma unroll
                for (int i = 0; i < DB; ++i) Xs[(kb + i) * SMEM_CB + g.t] = z[i];
            }
            g.sync();
            if (kb > 0) {
                float acc[QR][4];
#pragma unroll
                for (int q = 0; q < QR; ++q)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[q][c] = 0.f;
                for (int k = kb; k < ke; ++k) {
                    const float4 z = *reinterpret_cast<const float4*>(Xs + k * SMEM_CB + 4 * tx);
#pragma unroll
                    for (int q = 0; q < QR; ++q) {
                        const int r = ty + TY * q;
                        const float u = r < kb ? L[r * LD + k] : 0.f;
                        acc[q][0] = fmaf(u, z.x, acc[q][0]);
                        acc[q][1] = fmaf(u, z.y, acc[q][1]);
                        acc[q][2] = fmaf(u, z.z, acc[q][2]);
                        acc[q][3] = fmaf(u, z.w, acc[q][3]);
                    }
                }
#pragma unroll
                for (int q = 0; q < QR; ++q) {
                    const int r = ty + TY * q;
                    if (r < kb) {
                        float4* px = reinterpret_cast<float4*>(Xs + r * SMEM_CB + 4 * tx);
                        float4 v = *px;
                        v.x -= acc[q][0]; v.y -= acc[q][1]; v.z -= acc[q][2]; v.w -= acc[q][3];
                        *px = v;
                    }
                }
                g.sync();
            }
        }
        for (int r = rr; r < M; r += RPP)
            if (on) X[(size_t)r * ldx + c0 + cc] = Xs[r * SMEM_CB + cc];
        g.sync();
    }
    return ok;
}


// ---------------------------------------------------------------- dispatch
// One-warp groups use the register versions (they need a small shared
// scratch: `wsc`, at least 2 * (max(M, N) + 3) floats); wider groups use the
// step-synchronous versions.
template <int M, int NT>
__device__ __forceinline__ bool chol(const Grp<NT>& g, float* L, int ld, float* dinv, float* wsc)
{
    if constexpr (NT == 32 && M <= 32) return chol_warp<M>(g.t, L, ld, dinv, wsc);
    else return chol_generic<M, NT>(g, L, ld, dinv);
}

template <int M, int NC, int NT>
__device__ __forceinline__ void trsm_lower(const Grp<NT>& g, const float* L, int ld,
                                           const float* dinv, float* X, int ldx)
{
    if constexpr (NT == 32 && M <= 32) trsm_lower_warp<M, NC>(g.t, L, ld, dinv, X, ldx);
    else trsm_lower_generic<M, NC, NT>(g, L, ld, dinv, X, ldx);
}

template <int M, int NC, int NT>
__device__ __forceinline__ void trsm_lower_t(const Grp<NT>& g, const float* L, int ld,
                                             const float* dinv, float* X, int ldx)
{
    if constexpr (NT == 32 && M <= 32) trsm_lower_t_warp<M, NC>(g.t, L, ld, dinv, X, ldx);
    else trsm_lower_t_generic<M, NC, NT>(g, L, ld, dinv, X, ldx);
}

template <int N, int NR, int NT>
__device__ __forceinline__ bool gj_solve(const Grp<NT>& g, float* G, int ld, float* wsc)
{
    if constexpr (NT == 32 && N <= 32 && (N + NR + 31) / 32 <= 2) return gj_warp<N, NR>(g.t, G, ld, wsc);
    else return gj_solve_generic<N, NR, NT>(g, G, ld, wsc);
}

}  // namespace pdl
