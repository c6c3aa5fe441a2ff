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
    __device__ __forceinline__ void sync() const {
        if constexpr (NT == 32) {
            __syncwarp();
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

// out[R][C] = D + sgn * op(A) op(B)   (D == nullptr: no addend)
// op(A)(r,l) = TA ? A[l*lda + r] : A[r*lda + l];  op(B)(l,c) likewise.
// out must not alias A or B; it may alias D.
template <int R, int C, int K, bool TA, bool TB, int NT, bool SYNC = true>
__device__ __forceinline__ void mm(const Grp<NT>& g, float* out, int ldo,
                                   const float* A, int lda, const float* B, int ldb,
                                   const float* D = nullptr, int ldd = 0, float sgn = 1.f)
{
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
#pragma unroll
        for (int i = 0; i < RT; ++i) {
            const int r = r0 + i;
            if (R % RT != 0 && r >= R) continue;
#pragma unroll
            for (int j = 0; j < CT; ++j) {
                const int c = c0 + j;
                if (C % CT != 0 && c >= C) continue;
                float v = sgn * acc[i][j];
                if (D) v += D[r * ldd + c];
                out[r * ldo + c] = v;
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
// [Mx | RHS] (Mx is N x N in columns 0..N-1, NR right-hand sides after it).
// On exit columns N..N+NR-1 hold Mx^{-1} RHS.  Returns false (uniformly) if
// a pivot is zero or not finite.
template <int N, int NR, int NT>
__device__ bool gj_solve_generic(const Grp<NT>& g, float* G, int ld)
{
    constexpr int W = N + NR;
    bool ok = true;
    for (int k = 0; k < N; ++k) {
        int piv = k;
        float best = fabsf(G[k * ld + k]);
        for (int i = k + 1; i < N; ++i) {
            const float v = fabsf(G[i * ld + k]);
            if (v > best) { best = v; piv = i; }
        }
        ok = ok && (best > 1e-30f) && isfinite(best);
        if (piv != k) {  // uniform: every thread saw the same column
            g.sync();
            for (int j = k + g.t; j < W; j += NT) {
                const float a = G[k * ld + j];
                G[k * ld + j] = G[piv * ld + j];
                G[piv * ld + j] = a;
            }
            g.sync();
        }
        const float inv = 1.f / G[k * ld + k];
        for (int j = k + 1 + g.t; j < W; j += NT) G[k * ld + j] *= inv;
        g.sync();
        const int cols = W - k - 1;
        for (int e = g.t; e < (N - 1) * cols; e += NT) {
            const int ii = e / cols;
            const int i = ii + (ii >= k ? 1 : 0);
            const int j = k + 1 + e % cols;
            G[i * ld + j] -= G[i * ld + k] * G[k * ld + j];
        }
        g.sync();
    }
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
    else return gj_solve_generic<N, NR, NT>(g, G, ld);
}

}  // namespace pdl
