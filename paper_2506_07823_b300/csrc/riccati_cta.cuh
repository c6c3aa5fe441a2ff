// riccati_cta.cuh -- the sequential Riccati recursion (Eq. lqr, Sec. II-C)
// for mid-size LQ problems (n + m < 64: the whole-body-sized n = 36, m = 24,
// and n = m = 24) with one 128-thread CTA per instance.
//
// One backward step from V_{k+1} = (P', p') computes, in this order,
//   Y = P' [A | B],  w = P' c + p',  t = A^T p'                    (product 1)
//   [G | H | h] = [R | S | r] + B^T [P'B | P'A | w]                 (product 2)
//   G^-1 [H | h] by Gauss-Jordan elimination of the SPD G without pivoting;
//   K = -G^-1 H,  k = -G^-1 h
//   [Abar | bbar] = [A | c] + B [K | k]                             (product 4)
//   P = Q + (P'A)^T Abar + S^T K,  p = q + t + (P'A)^T bbar + S^T k (product 5)
// The last line is Eq. lqr's P = Q + A^T P' A + K^T H, p = q + A^T (p' + P'c)
// + K^T h rewritten with H = S + B^T P'A and P' = P'^T: K^T H = (P'A)^T B K
// + S^T K, so that neither H nor a second copy of B K is needed.  P is
// computed on its upper triangle and mirrored (exactly symmetric).
//
// Every product is register-tiled: a thread owns a tile of TR rows x 4
// columns of the output and streams the contraction dimension k, reading
// the left operand k-major (row k of L^T, TR consecutive floats) and row k of
// the right operand (one float4) from shared memory.  The elimination keeps
// one column of [G | H | h] per pair of threads (NU / 2 rows each) in
// registers and exchanges the pivot row and column through shared memory,
// one barrier per pivot.
// The forward rollout reuses the chunk rollout of the scan kernels on the
// stored K, k, P, p, Abar, bbar.
#pragma once

#include "kkt_scan.cuh"

namespace pdl {

constexpr int kRcThreads = 128;

template <int NX, int NU>
struct RicCtaL {
    static constexpr int YC = NX + NU;                  // columns of Y = P'[A | B]
    static constexpr int GC = round4(NU + NX + 1);      // columns of [G | H | h] (and pad)
    // one stage's inputs (two banks: the next stage is copied in meanwhile)
    static constexpr int A = 0;                         // A, then Abar  (NX x NX)
    static constexpr int Bm = A + NX * NX;              // B             (NX x NU)
    static constexpr int S = Bm + NX * NU;              // S             (NU x NX), if given
    static constexpr int c = S + NU * NX;               // c, then bbar  (NX)
    static constexpr int q = c + round4(NX);
    static constexpr int r = q + round4(NX);
    static constexpr int IN = r + round4(NU);           // floats of one bank
    // work areas after the two banks
    static constexpr int Bt = 2 * IN;                   // B^T           (NU x NX)
    static constexpr int V = Bt + NU * NX;              // P' then P (NX x NX), p' then p (NX)
    static constexpr int Y = V + NX * NX + round4(NX);  // P'[A | B]     (NX x YC)
    static constexpr int w = Y + NX * YC;               // P'c + p'      (NX)
    static constexpr int t = w + round4(NX);            // A^T p'        (NX)
    static constexpr int G = t + round4(NX);            // [G | H | h]   (NU x GC)
    static constexpr int XR = G + NU * GC;              // pivot rows    (2 x GC)
    static constexpr int XC = XR + 2 * GC;              // pivot columns (2 x round4(NU))
    static constexpr int SIZE = XC + 2 * round4(NU);
    static constexpr size_t BYTES = sizeof(float) * SIZE;
    static_assert(NX % 4 == 0 && NU % 4 == 0 && NU + NX + 1 <= 64,
                  "one column of [G | H | h] per pair of threads");
    static_assert(NX % 6 == 0 && NU % 8 == 0, "tile shapes");
};

// TR consecutive floats at p (p is 8-byte aligned when TR is even and
// 16-byte aligned when TR % 4 == 0).
template <int TR>
__device__ __forceinline__ void ld_vec(float (&v)[TR], const float* p)
{
    if constexpr (TR % 4 == 0) {
#pragma unroll
        for (int a = 0; a < TR; a += 4) {
            const float4 x = *reinterpret_cast<const float4*>(p + a);
            v[a] = x.x; v[a + 1] = x.y; v[a + 2] = x.z; v[a + 3] = x.w;
        }
    } else if constexpr (TR % 2 == 0) {
#pragma unroll
        for (int a = 0; a < TR; a += 2) {
            const float2 x = *reinterpret_cast<const float2*>(p + a);
            v[a] = x.x; v[a + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int a = 0; a < TR; ++a) v[a] = p[a];
    }
}

// acc[a][b] += sum_{k < KD} Lt[k * ldl + a] * R[k * ldr + b]   (a < TR, b < 4)
template <int TR, int KD>
__device__ __forceinline__ void tile_acc(float (&acc)[TR][4], const float* Lt, int ldl,
                                         const float* R, int ldr)
{
#pragma unroll 4
    for (int k = 0; k < KD; ++k) {
        float l[TR];
        ld_vec<TR>(l, Lt + k * ldl);
        const float4 b = *reinterpret_cast<const float4*>(R + k * ldr);
#pragma unroll
        for (int a = 0; a < TR; ++a) {
            acc[a][0] = fmaf(l[a], b.x, acc[a][0]);
            acc[a][1] = fmaf(l[a], b.y, acc[a][1]);
            acc[a][2] = fmaf(l[a], b.z, acc[a][2]);
            acc[a][3] = fmaf(l[a], b.w, acc[a][3]);
        }
    }
}

// acc[a] += sum_{k < KD} Lt[k * ldl + a] * v[k * ldv]   (a < TR): a TR-row
// slice of a matrix-vector product with the matrix read k-major
template <int TR, int KD>
__device__ __forceinline__ void col_acc(float (&acc)[TR], const float* Lt, int ldl, const float* v,
                                        int ldv)
{
#pragma unroll 4
    for (int k = 0; k < KD; ++k) {
        float l[TR];
        ld_vec<TR>(l, Lt + k * ldl);
        const float x = v[k * ldv];
#pragma unroll
        for (int a = 0; a < TR; ++a) acc[a] = fmaf(l[a], x, acc[a]);
    }
}

__device__ __forceinline__ float4 f4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}


// ------------------------------------------------------------ one stage
// Stage gs's A, B, c, q, r (and S) into the input bank `in`: one thread
// issues one bulk copy per array on the TMA engine, all completing on the
// bank's mbarrier (every array is contiguous per stage; sizes and offsets are
// multiples of 16 bytes and the base pointers are 16-byte aligned, checked
// at the boundary).
template <int NX, int NU>
struct RcBulk {
    static constexpr uint32_t A = NX * NX * 4, B = NX * NU * 4, S = NU * NX * 4, c = NX * 4,
                              q = NX * 4, r = NU * 4;
    static_assert(A % 16 == 0 && B % 16 == 0 && c % 16 == 0 && r % 16 == 0, "bulk copy sizes");
};

template <int NX, int NU>
__device__ __forceinline__ void rc_load(float* in, uint64_t* mbar, const KktArgs& a, int64_t gs, bool has_S)
{
    using L = RicCtaL<NX, NU>;
    using Z = RcBulk<NX, NU>;
    mbar_arrive_expect_tx(mbar, Z::A + Z::B + Z::c + Z::q + Z::r + (has_S ? Z::S : 0u));
    bulk_g2s(in + L::A, a.A + gs * NX * NX, Z::A, mbar);
    bulk_g2s(in + L::Bm, a.B + gs * NX * NU, Z::B, mbar);
    if (has_S) bulk_g2s(in + L::S, a.S + gs * NU * NX, Z::S, mbar);
    bulk_g2s(in + L::c, a.c + gs * NX, Z::c, mbar);
    bulk_g2s(in + L::q, a.q + gs * NX, Z::q, mbar);
    bulk_g2s(in + L::r, a.r + gs * NU, Z::r, mbar);
}

// Product 1: Y = P'[A | B] (6 x 4 tiles), w = P'c + p', t = A^T p', and the
// transposed copy of B used by product 4.
template <int NX, int NU>
__device__ __forceinline__ void rc_product1(float* sm, const float* in, int t)
{
    using L = RicCtaL<NX, NU>;
    constexpr int RG = NX / 6, CG = L::YC / 4, TILES = RG * CG, VT = NX / 4;
    const float* P1 = sm + L::V;
    const float* p1 = sm + L::V + NX * NX;
    for (int task = t; task < TILES + 2 * VT; task += kRcThreads) {
        if (task < TILES) {
            const int i0 = 6 * (task / CG), j0 = 4 * (task % CG);
            const float* R = j0 < NX ? in + L::A + j0 : in + L::Bm + (j0 - NX);
            const int ldr = j0 < NX ? NX : NU;
            float acc[6][4] = {};
            tile_acc<6, NX>(acc, P1 + i0, NX, R, ldr);
#pragma unroll
            for (int a = 0; a < 6; ++a)
                st4(sm + L::Y + (i0 + a) * L::YC + j0, acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
        } else if (task < TILES + VT) {
            const int i0 = 4 * (task - TILES);
            float acc[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[a] = p1[i0 + a];
            col_acc<4, NX>(acc, P1 + i0, NX, in + L::c, 1);
            st4(sm + L::w + i0, acc[0], acc[1], acc[2], acc[3]);
        } else {
            const int i0 = 4 * (task - TILES - VT);
            float acc[4] = {};
            col_acc<4, NX>(acc, in + L::A + i0, NX, p1, 1);
            st4(sm + L::t + i0, acc[0], acc[1], acc[2], acc[3]);
        }
    }
    for (int e = t; e < NX * NU; e += kRcThreads) {
        const int i = e / NU, j = e % NU;
        sm[L::Bt + j * NX + i] = in[L::Bm + e];
    }
}

// Product 2: [G | H | h] = [R | S | r] + B^T [P'B | P'A | w] (4 x 4 tiles);
// R is read from global memory (issued before the contraction, added after
// it), the pad columns are set to zero.
template <int NX, int NU>
struct RcP2 {
    static constexpr int RG = NU / 4, CG = (NU + NX) / 4, TILES = RG * CG, TASKS = TILES + NU / 4;
};

template <int NX, int NU>
__device__ __forceinline__ void rc_product2(float* sm, const float* in, const KktArgs& a, int64_t gs,
                                            bool has_S, int task)
{
    using L = RicCtaL<NX, NU>;
    using T = RcP2<NX, NU>;
    float* Gm = sm + L::G;
    if (task < T::TILES) {
        const int i0 = 4 * (task / T::CG), j0 = 4 * (task % T::CG);
        float4 add[4];
        if (j0 < NU) {
            const float* Rg = a.R + gs * NU * NU + i0 * NU + j0;
#pragma unroll
            for (int r = 0; r < 4; ++r) add[r] = __ldg(reinterpret_cast<const float4*>(Rg + r * NU));
        } else if (has_S) {
#pragma unroll
            for (int r = 0; r < 4; ++r) add[r] = f4(in + L::S + (i0 + r) * NX + (j0 - NU));
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) add[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float acc[4][4] = {};
        const float* R = j0 < NU ? sm + L::Y + NX + j0 : sm + L::Y + (j0 - NU);
        tile_acc<4, NX>(acc, in + L::Bm + i0, NU, R, L::YC);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            acc[r][0] += add[r].x; acc[r][1] += add[r].y; acc[r][2] += add[r].z; acc[r][3] += add[r].w;
            st4(Gm + (i0 + r) * L::GC + j0, acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
        }
    } else {
        const int i0 = 4 * (task - T::TILES);
        float acc[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] = in[L::r + i0 + r];
        col_acc<4, NX>(acc, in + L::Bm + i0, NU, sm + L::w, 1);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float* row = Gm + (i0 + r) * L::GC;
            row[NU + NX] = acc[r];
            for (int j = NU + NX + 1; j < L::GC; ++j) row[j] = 0.f;
        }
    }
}

// Gauss-Jordan elimination of [G | H | h] (G SPD, no pivoting): thread t owns
// column t mod 64 in rows [NU/2 (t / 64), NU/2 (t / 64) + NU/2) in
// registers; before pivot k the exchange buffers hold row k and column k of
// the current matrix (double-buffered by the parity of k, so one barrier per
// pivot).  Writes K = -G^-1 H and k = -G^-1 h over the H and h columns (in
// shared memory and to stage gs in global memory); returns whether every
// pivot was positive (uniform over the CTA).
template <int NX, int NU>
__device__ __forceinline__ bool rc_solve(float* sm, const KktArgs& a, int64_t gs, int t)
{
    using L = RicCtaL<NX, NU>;
    constexpr int RPT = NU / 2, XCL = round4(NU);
    float* Gm = sm + L::G;
    float* XR = sm + L::XR;
    float* XC = sm + L::XC;
    const int j = t & 63, hh = t >> 6;
    const bool own = j < L::GC;
    float v[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) v[r] = own ? Gm[(hh * RPT + r) * L::GC + j] : 0.f;
    if (hh == 0 && own) XR[j] = v[0];
    if (j == 0) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) XC[hh * RPT + r] = v[r];
    }
    __syncthreads();
    bool spd = true;
#pragma unroll
    for (int k = 0; k < NU; ++k) {
        const int b = k & 1;
        const float d = XR[b * L::GC + k];
        spd = spd && d > 0.f;
        const float s = (own ? XR[b * L::GC + j] : 0.f) * rcp_approx(d);
        float cc[RPT];
        ld_vec<RPT>(cc, XC + b * XCL + hh * RPT);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            if (r == k % RPT && hh == k / RPT) v[r] = s;
            else v[r] = fmaf(-cc[r], s, v[r]);
        }
        if (k + 1 < NU) {
            const int bn = b ^ 1;
            if (hh == (k + 1) / RPT && own) XR[bn * L::GC + j] = v[(k + 1) % RPT];
            if (j == k + 1) {
#pragma unroll
                for (int r = 0; r < RPT; ++r) XC[bn * XCL + hh * RPT + r] = v[r];
            }
            __syncthreads();
        }
    }
    if (own && j >= NU && j <= NU + NX) {
        const int jj = j - NU;
        float* out = jj < NX ? a.K + gs * NU * NX + jj : a.k + gs * NU;
        const int ld = jj < NX ? NX : 1;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int i = hh * RPT + r;
            Gm[i * L::GC + j] = -v[r];
            out[i * ld] = -v[r];
        }
    }
    return spd;
}

// Product 4: [Abar | bbar] = [A | c] + B [K | k] in place of A and c (4 x 4
// tiles), also stored to stage gs in global memory.
template <int NX, int NU>
struct RcP4 {
    static constexpr int RG = NX / 4, CG = NX / 4, TILES = RG * CG, TASKS = TILES + NX / 4;
};

template <int NX, int NU>
__device__ __forceinline__ void rc_product4(float* sm, float* in, const KktArgs& a, int64_t gs, int task)
{
    using L = RicCtaL<NX, NU>;
    using T = RcP4<NX, NU>;
    const float* Km = sm + L::G + NU;
    if (task < T::TILES) {
        const int i0 = 4 * (task / T::CG), j0 = 4 * (task % T::CG);
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float4 v = f4(in + L::A + (i0 + r) * NX + j0);
            acc[r][0] = v.x; acc[r][1] = v.y; acc[r][2] = v.z; acc[r][3] = v.w;
        }
        tile_acc<4, NU>(acc, sm + L::Bt + i0, NX, Km + j0, L::GC);
        float* Ag = a.Abar + gs * NX * NX;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            st4(in + L::A + (i0 + r) * NX + j0, acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
            st4(Ag + (i0 + r) * NX + j0, acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
        }
    } else {
        const int i0 = 4 * (task - T::TILES);
        float acc[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] = in[L::c + i0 + r];
        col_acc<4, NU>(acc, sm + L::Bt + i0, NX, Km + NX, L::GC);
        st4(in + L::c + i0, acc[0], acc[1], acc[2], acc[3]);
        st4(a.bbar + gs * NX + i0, acc[0], acc[1], acc[2], acc[3]);
    }
}

// Product 5: P = Q + (P'A)^T Abar + S^T K on the upper-triangle 4 x 4 tiles,
// mirrored; p = q + A^T p' + (P'A)^T bbar + S^T k.  Into the value-function
// area and to stage gs in global memory.  Q is read from global memory
// (issued before the contraction, added after it).
template <int NX, int NU>
struct RcP5 {
    static constexpr int RG = NX / 4, UT = RG * (RG + 1) / 2, TASKS = UT + NX / 4;
};

template <int NX, int NU>
__device__ __forceinline__ void rc_product5(float* sm, const float* in, const KktArgs& a, int64_t gs,
                                            bool has_S, int task)
{
    using L = RicCtaL<NX, NU>;
    using T = RcP5<NX, NU>;
    const float* Km = sm + L::G + NU;
    float* P = sm + L::V;
    if (task < T::UT) {
        // task -> (rg, cg) with rg <= cg, row by row of the upper triangle
        int rg = 0, rem = task;
        while (rem >= T::RG - rg) { rem -= T::RG - rg; ++rg; }
        const int i0 = 4 * rg, j0 = 4 * (rg + rem);
        float4 add[4];
        const float* Qg = a.Q + gs * NX * NX + i0 * NX + j0;
#pragma unroll
        for (int r = 0; r < 4; ++r) add[r] = __ldg(reinterpret_cast<const float4*>(Qg + r * NX));
        float acc[4][4] = {};
        tile_acc<4, NX>(acc, sm + L::Y + i0, L::YC, in + L::A + j0, NX);
        if (has_S) tile_acc<4, NU>(acc, in + L::S + i0, NX, Km + j0, L::GC);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            acc[r][0] += add[r].x; acc[r][1] += add[r].y; acc[r][2] += add[r].z; acc[r][3] += add[r].w;
        }
        if (i0 == j0) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = r + 1; c < 4; ++c) {
                    const float m = 0.5f * (acc[r][c] + acc[c][r]);
                    acc[r][c] = m;
                    acc[c][r] = m;
                }
        }
        float* Pg = a.P + gs * NX * NX;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            st4(P + (i0 + r) * NX + j0, acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
            st4(Pg + (i0 + r) * NX + j0, acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
        }
        if (i0 != j0) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                st4(P + (j0 + c) * NX + i0, acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
                st4(Pg + (j0 + c) * NX + i0, acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
            }
        }
    } else {
        const int i0 = 4 * (task - T::UT);
        float acc[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] = in[L::q + i0 + r] + sm[L::t + i0 + r];
        col_acc<4, NX>(acc, sm + L::Y + i0, L::YC, in + L::c, 1);
        if (has_S) col_acc<4, NU>(acc, in + L::S + i0, NX, Km + NX, L::GC);
        st4(P + NX * NX + i0, acc[0], acc[1], acc[2], acc[3]);
        st4(a.p + gs * NX + i0, acc[0], acc[1], acc[2], acc[3]);
    }
}

// ------------------------------------------------------------ kernel
// One CTA of 128 threads per instance (slot blockIdx.x of the longest-first
// order): the terminal value function, N backward steps (stage k - 1's
// inputs are bulk-copied into the other bank while stage k is processed;
// a copy that does not land within the bounded wait ends the instance with
// status TIMEOUT), then
// the forward rollout dx_{k+1} = Abar_k dx_k + bbar_k with du_k = K_k dx_k +
// k_k and dlam_k = P_k dx_k + p_k.  Status: NOT_SPD if a pivot of some G_k
// was not positive, NONFINITE if an output is not finite.
template <int NX, int NU>
__global__ void __launch_bounds__(kRcThreads, 4) riccati_cta_kernel(const __grid_constant__ KktArgs a)
{
    using L = RicCtaL<NX, NU>;
    extern __shared__ __align__(16) float sm[];
    __shared__ uint64_t mbar[2];   // one per input bank
    const int t = threadIdx.x;
    const int slot = blockIdx.x;
    if (slot >= a.count) return;
    const int inst = a.order ? a.order[slot] : slot;
    const int N = a.N[inst];
    const int64_t off = a.off[inst];
    const bool has_S = a.S != nullptr;
    // test switch: no bulk copy is issued, so the first bounded wait runs out
    const bool issue = (a.dbg & PDILQR_DEBUG_BULK_SKIP_ISSUE) == 0;
    if (t == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (t == 0 && N > 0 && issue)
        rc_load<NX, NU>(sm + ((N - 1) & 1) * L::IN, &mbar[(N - 1) & 1], a, off + N - 1, has_S);
    {
        const int64_t gN = off + N;
        for (int e = t; e < NX * NX / 4; e += kRcThreads) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(a.Q + gN * NX * NX) + e);
            reinterpret_cast<float4*>(sm + L::V)[e] = v;
            reinterpret_cast<float4*>(a.P + gN * NX * NX)[e] = v;
        }
        for (int i = t; i < NX; i += kRcThreads) {
            const float v = a.q[gN * NX + i];
            sm[L::V + NX * NX + i] = v;
            a.p[gN * NX + i] = v;
        }
        for (int e = t; e < NU * NX; e += kRcThreads) a.K[gN * NU * NX + e] = 0.f;
        for (int i = t; i < NU; i += kRcThreads) a.k[gN * NU + i] = 0.f;
    }
    bool spd = true, timed_out = false;
    uint32_t phase = 0;   // bit b: the parity bank b's next wait expects
    for (int k = N - 1; k >= 0; --k) {
        const int64_t gs = off + k;
        const int b = k & 1;
        float* in = sm + b * L::IN;
        // stage k's copies have landed (bounded wait, one verdict for the CTA)
        const bool got = mbar_wait_bounded(&mbar[b], (phase >> b) & 1u, kTcWaitNs);
        // the other bank (stage k + 1's) is free once every thread is here;
        // its generic-proxy writes (Abar, bbar in place) are ordered before
        // the bulk copies that overwrite it
        fence_proxy_async_smem();
        if (__syncthreads_or(got ? 0 : 1)) {
            // the copies of bank b (the only ones in flight) get a second
            // bounded wait before the CTA gives up its shared memory
            mbar_wait_bounded(&mbar[b], (phase >> b) & 1u, kTcDrainNs);
            timed_out = true;
            break;
        }
        phase ^= 1u << b;
        if (t == 0 && k > 0 && issue) rc_load<NX, NU>(sm + (b ^ 1) * L::IN, &mbar[b ^ 1], a, gs - 1, has_S);
        rc_product1<NX, NU>(sm, in, t);
        __syncthreads();
        for (int task = t; task < RcP2<NX, NU>::TASKS; task += kRcThreads)
            rc_product2<NX, NU>(sm, in, a, gs, has_S, task);
        __syncthreads();
        spd = rc_solve<NX, NU>(sm, a, gs, t) && spd;
        __syncthreads();
        for (int task = t; task < RcP4<NX, NU>::TASKS; task += kRcThreads)
            rc_product4<NX, NU>(sm, in, a, gs, task);
        __syncthreads();
        for (int task = t; task < RcP5<NX, NU>::TASKS; task += kRcThreads)
            rc_product5<NX, NU>(sm, in, a, gs, has_S, task);
    }
    if (timed_out) {
        if (t == 0) a.status[inst] = ST_TIMEOUT;
        return;
    }
    __syncthreads();
    // forward rollout from dx_0 = s over the stored stages (the global stores
    // of this CTA are visible to its own later loads after the barrier)
    using RL = RollL<NX, NU>;
    static_assert(2 * round4(NX) + 2 * RL::SIZE <= L::SIZE, "rollout buffers fit");
    float* x = sm;
    float* xn = sm + round4(NX);
    float* rb = sm + 2 * round4(NX);
    __threadfence_block();
    for (int i = t; i < NX; i += kRcThreads) x[i] = a.s[(int64_t)inst * NX + i];
    __syncthreads();
    const Grp<kRcThreads> g{t, 0};
    const bool fin = rollout_chunk<NX, NU, kRcThreads>(g, x, xn, rb, a, off, N, 0, N + 1);
    const bool bad_fin = __syncthreads_or(fin ? 0 : 1) != 0;
    if (t == 0) a.status[inst] = bad_fin ? ST_NONFINITE : (spd ? ST_OK : ST_NOT_SPD);
}

}  // namespace pdl
