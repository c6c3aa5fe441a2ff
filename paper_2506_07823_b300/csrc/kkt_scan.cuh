// kkt_scan.cuh -- LQ KKT solve of one primal-dual iLQR step on the GPU.
//
// Two solvers share the stage-level building blocks below:
//
//  * kkt_scan_kernel  -- the parallel associative scan of Sec. II-D.  One CTA
//    owns one instance; its W warps split the N+1 stages into W contiguous
//    chunks.  The reverse scan is a reduce-then-scan:
//      phase 1  middle chunks fold their CVF elements (Eq. initialization)
//               with the combine of Eq. (combination_rule) into one aggregate
//               per chunk, while the last chunk runs the value-function
//               recursion from the terminal cost;
//      phase 2  a Hillis-Steele suffix scan over the chunk aggregates gives
//               the value function (P, p) at every chunk boundary;
//      phase 3  every chunk walks its stages backwards from its boundary
//               value function: e_k (x) V_{k+1} is evaluated in its Riccati
//               form (Eq. lqr), which also yields the policy K_k, k_k of the
//               "one pass in parallel" recovery, and the chunk's closed-loop
//               affine map (Abar, bbar) of Eq. (controlled_dynamics);
//      phase 4  the trajectory scan: the chunk affine maps are composed from
//               dx_0, then each chunk rolls dx, du and dlam = P dx + p out.
//  * riccati_kernel   -- the sequential Riccati recursion (Eq. lqr) and
//    forward rollout, one warp per instance: the comparator.
//
// The combine uses the corrected rule (typos of the printed rule fixed):
//   M = I + C1 P2,
//   A = A2 M^-1 A1,            b = A2 M^-1 (b1 - C1 p2) + b2,
//   C = A2 M^-1 C1 A2^T + C2,  P = (M^-1 A1)^T P2 A1 + P1,
//   p = (M^-1 A1)^T (p2 + P2 b1) + p1,
// with M^-1 applied by Gauss-Jordan elimination with partial pivoting (one
// warp: M^-1 itself from [M | I], then products).  The SPD systems of the
// element build (R) and the Riccati step (G) are solved by elimination
// without pivoting, whose positive pivots are the SPD test.
#pragma once

#include "dev_linalg.cuh"
#include "pdilqr.h"

namespace pdl {

// Status codes written per instance (the C ABI's pdilqr_status values).
enum : int32_t {
    ST_OK = PDILQR_OK,
    ST_INVALID_ARG = PDILQR_E_INVALID_ARG,
    ST_NOT_SPD = PDILQR_E_NOT_SPD,
    ST_SINGULAR = PDILQR_E_SINGULAR,
    ST_NONFINITE = PDILQR_E_NONFINITE,
    ST_TIMEOUT = PDILQR_E_TIMEOUT
};
static_assert(ST_INVALID_ARG == 1 && ST_NONFINITE == 4 && ST_TIMEOUT == 5,
              "per-instance status words carry the C ABI's codes");

struct KktArgs {
    const float *A, *B, *c, *Q, *R, *S, *q, *r;  // LQ data; S may be null (S = 0)
    const float* s;                              // [count][n] dx_0
    float *dx, *du, *dlam;                       // outputs, N+1 stage slots
    float *K, *k, *P, *p;                        // policy and value function per stage
    float *Abar, *bbar;                          // closed-loop maps per stage
    const int32_t* N;                            // [count] horizon
    const int64_t* off;                          // [count] first stage slot
    const int32_t* order;                        // [count] CTA -> instance (longest first)
    int32_t* status;                             // [count]
    int count;
    float* gws;                                  // per-CTA work areas in global memory
                                                 // (sizes whose areas exceed shared memory)
    int dbg;                                     // test switches (PDILQR_DEBUG_*), normally 0
    int m64 = 0;                                 // 1: the combines eliminate M = I + C1 P2
                                                 // in FP64 (n = 36; gj_solve_f64)
    unsigned* sbar = nullptr;                    // [count] phase counters of the split scan
};

// ------------------------------------------------------------------ layouts
template <int NX, int NU>
struct StageL {  // one stage of LQ data staged in shared memory (every block
                 // starts on a 16-byte boundary); IN is the model-input area
                 // of sources that linearise on the fly
    static constexpr int A = 0, B = round4(A + NX * NX), Q = round4(B + NX * NU),
                         R = round4(Q + NX * NX), S = round4(R + NU * NU),
                         c = round4(S + NU * NX), q = round4(c + NX), r = round4(q + NX),
                         IN = round4(r + NU),
                         SIZE = round4(IN + 5 * round4(NX) + 2 * round4(NU) + round4(NX / 12 + 1));
};

template <int NX>
struct ElemL {  // CVF element (A, C, b, P, p); a value function uses P, p only,
                // which are contiguous so that it copies as one block
    static constexpr int A = 0, C = NX * NX, b = 2 * NX * NX, P = 2 * NX * NX + NX,
                         p = 3 * NX * NX + NX, SIZE = round4(3 * NX * NX + 2 * NX);
};

// (Wk: small scratch of the one-warp factorisations, 3 (dim + 1) floats)
template <int NX, int NU>
struct BuildL {  // scratch of the element build
    static constexpr int Lr = 0, dinv = Lr + NU * NU, Z = round4(dinv + NU),
                         Y = Z + NU * NX, Wk = round4(Y + NU * (NX + 1)),
                         SIZE = round4(Wk + 3 * (NU + 1));
};

template <int NX>
struct CombL {  // scratch of a combine
    static constexpr int LDG = 3 * NX + 1;
    static constexpr int G = 0, T = round4(NX * LDG), U = T + NX * NX, w = U + NX * NX,
                         Wk = round4(w + NX), SIZE0 = round4(Wk + 3 * (NX + 1));
    // one-warp full combine through M^-1: [M | I] (T reuses its area once
    // M^-1 has been applied), M^-1 A1, M^-1 C1, b1 - C1 p2 and M^-1 of it
    static constexpr int LDI = 2 * NX;
    static constexpr int GI = 0, XA = round4(NX * LDI), XC = XA + NX * NX, UI = XC + NX * NX,
                         wI = UI + NX * NX, xb = round4(wI + NX), vb = round4(xb + NX),
                         WkI = round4(vb + NX), SIZE1 = round4(WkI + 3 * (NX + 1));
    static constexpr int SIZE = SIZE0 > SIZE1 ? SIZE0 : SIZE1;
};

// SPD systems of at least this many rows are factored in a shared-memory
// factor buffer when the unit has one (smaller ones are eliminated in place).
constexpr int kSmemFactorRows = 96;

// One-warp fast paths: SPD solves by Gauss-Jordan without pivoting when
// [G | H | h] fits one column per lane; the full combine through M^-1 when
// [M | I] does.
template <int NX, int NU, int NT>
struct WarpPath {
    static constexpr bool spd = NT == 32 && NU + NX + 1 <= 32;
    static constexpr bool inv = NT == 32 && 2 * NX <= 32;
    // groups wider than one warp: SPD solves by the generic elimination
    static constexpr bool spd_wide = NT > 32;
};

template <int NX, int NU>
struct RicL {  // scratch of one Riccati step; Y2 = G^-1 [H | h] reuses the
               // area of P'B and P'c + p', which are dead once G and h exist,
               // and Abar the area of P'A; Abar and bbar stay there for the caller
    static constexpr int PB = 0, w = PB + NX * NU, Y2 = 0,
                         R0 = NX * NU + NX > NU * (NX + 1) ? NX * NU + NX : NU * (NX + 1),
                         PA = round4(R0), Ab = PA, G = round4(PA + NX * NX), dinv = G + NU * NU,
                         Y = round4(dinv + NU), Wk = round4(Y + NU * (NX + 1)),
                         bb = round4(Wk + 3 * (NU + 1)), SIZE = round4(bb + NX);
};

// Copy COUNT floats (shared or work-area memory) to global memory, 16 bytes
// at a time when both ends are 16-byte aligned (uniform over the group).
template <int COUNT, int NT>
__device__ __forceinline__ void store_out(int t, float* dst, const float* src)
{
    if constexpr (COUNT % 4 == 0) {
        if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0) {
            for (int e = t; e < COUNT / 4; e += NT)
                reinterpret_cast<float4*>(dst)[e] = reinterpret_cast<const float4*>(src)[e];
            return;
        }
    }
    for (int e = t; e < COUNT; e += NT) dst[e] = src[e];
}

// ------------------------------------------------------------ stage loading
// All blocks of one stage are copied asynchronously and waited for once.
template <int NX, int NU, int NT>
__device__ __forceinline__ void load_stage(const Grp<NT>& g, float* st, const KktArgs& a,
                                           int64_t gs, bool terminal)
{
    using L = StageL<NX, NU>;
    stage_copy<NX * NX, NT, true>(g.t, st + L::Q, a.Q + gs * NX * NX);
    stage_copy<NX, NT, true>(g.t, st + L::q, a.q + gs * NX);
    if (!terminal) {
        stage_copy<NX * NX, NT, true>(g.t, st + L::A, a.A + gs * NX * NX);
        stage_copy<NX * NU, NT, true>(g.t, st + L::B, a.B + gs * NX * NU);
        stage_copy<NU * NU, NT, true>(g.t, st + L::R, a.R + gs * NU * NU);
        stage_copy<NX, NT, true>(g.t, st + L::c, a.c + gs * NX);
        stage_copy<NU, NT, true>(g.t, st + L::r, a.r + gs * NU);
        if (a.S) stage_copy<NU * NX, NT, true>(g.t, st + L::S, a.S + gs * NU * NX);
    }
    cp_async_commit();
    cp_async_wait_all();
    g.sync();
}

// Source of LQ stages read from the caller's arrays.
struct LqSource {
    const float *A, *B, *c, *Q, *R, *S, *q, *r;
    __device__ explicit LqSource(const KktArgs& a)
        : A(a.A), B(a.B), c(a.c), Q(a.Q), R(a.R), S(a.S), q(a.q), r(a.r) {}
    template <int NX, int NU, int NT>
    __device__ __forceinline__ void load(const Grp<NT>& g, float* st, int64_t gs, bool terminal) const
    {
        KktArgs t;
        t.A = A; t.B = B; t.c = c; t.Q = Q; t.R = R; t.S = S; t.q = q; t.r = r;
        load_stage<NX, NU, NT>(g, st, t, gs, terminal);
    }
    // the caller's arrays are read again in the Riccati sweep: nothing to keep
    static constexpr bool kKeeps = false;
    template <int NX, int NU, int NT>
    __device__ __forceinline__ void keep(const Grp<NT>&, const float*, int64_t) const {}
    template <int NX, int NU, int NT>
    __device__ __forceinline__ void reload(const Grp<NT>& g, float* st, int64_t gs) const
    {
        load<NX, NU, NT>(g, st, gs, false);
    }
    __device__ __forceinline__ bool has_S() const { return S != nullptr; }
};

// ------------------------------------------------------------ element build
// e_k = (A - B R^-1 S, c - B R^-1 r, B R^-1 B^T, q - S^T R^-1 r, Q - S^T R^-1 S)
// (Eq. initialization); the terminal element is (0, 0, 0, q_N, Q_N).
template <int NX, int NU, int NT, bool FAC = false>
__device__ bool build_element(const Grp<NT>& g, const float* st, float* e, float* scr,
                              bool has_S, bool terminal)
{
    using L = StageL<NX, NU>;
    using E = ElemL<NX>;
    using S = BuildL<NX, NU>;
    if (terminal) {
        fill<NX, NX, NT, false>(g, e + E::A, NX, 0.f);
        fill<NX, NX, NT, false>(g, e + E::C, NX, 0.f);
        for (int i = g.t; i < NX; i += NT) { e[E::b + i] = 0.f; e[E::p + i] = st[L::q + i]; }
        copy<NX, NX, false, NT>(g, e + E::P, NX, st + L::Q, NX);
        return true;
    }
    float* Lr = scr + S::Lr;
    float* dinv = scr + S::dinv;
    float* Z = scr + S::Z;
    float* Y = scr + S::Y;
    constexpr int LDY = NX + 1;
    if constexpr (WarpPath<NX, NU, NT>::spd || WarpPath<NX, NU, NT>::spd_wide) {
        if (!has_S) {
            // [X | y] = R^-1 [B^T | r] in one elimination;  C = B X,  b = c - B y
            copy<NU, NX, true, NT, false>(g, Y, LDY, st + L::B, NU);
            for (int i = g.t; i < NU; i += NT) Y[i * LDY + NX] = st[L::r + i];
            bool ok;
            if constexpr (WarpPath<NX, NU, NT>::spd) {
                g.sync();
                ok = spd_solve_warp<NU, NX + 1>(g.t, st + L::R, NU, Y, LDY, Y, LDY, scr + S::Wk);
            } else {
                // large systems: the factorisation in the unit's factor buffer
                // (compiled only where the launch configuration has such a buffer)
                bool done = false;
                if constexpr (FAC) {
                    if (g.fb && g.fbn >= spd_smem_floats(NU)) {
                        g.sync();
                        ok = spd_solve_smem<NU, NX + 1, NT>(g, st + L::R, NU, Y, LDY, dinv);
                        done = true;
                    }
                }
                if (!done) {
                    copy<NU, NU, false, NT>(g, Lr, NU, st + L::R, NU);
                    ok = spd_solve_generic<NU, NX + 1, NT>(g, Lr, NU, Y, LDY, dinv);
                }
            }
            mm<NX, NX, NU, false, false, NT, false>(g, e + E::C, NX, st + L::B, NU, Y, LDY);
            mm<NX, 1, NU, false, false, NT, false>(g, e + E::b, 1, st + L::B, NU, Y + NX, LDY,
                                                   st + L::c, 1, -1.f);
            copy<NX, NX, false, NT, false>(g, e + E::A, NX, st + L::A, NX);
            copy<NX, NX, false, NT, false>(g, e + E::P, NX, st + L::Q, NX);
            for (int i = g.t; i < NX; i += NT) e[E::p + i] = st[L::q + i];
            g.sync();
            symmetrize<NX, NT>(g, e + E::C, NX);
            return ok;
        }
    }
    copy<NU, NU, false, NT, false>(g, Lr, NU, st + L::R, NU);
    copy<NU, NX, true, NT, false>(g, Z, NX, st + L::B, NU);   // Z = B^T
    if (has_S) copy<NU, NX, false, NT, false>(g, Y, LDY, st + L::S, NX);
    for (int i = g.t; i < NU; i += NT) Y[i * LDY + NX] = st[L::r + i];
    g.sync();
    const bool ok = chol<NU, NT>(g, Lr, NU, dinv, scr + S::Wk);
    trsm_lower<NU, NX, NT>(g, Lr, NU, dinv, Z, NX);             // Z = L^-1 B^T
    if (has_S) {
        trsm_lower<NU, NX + 1, NT>(g, Lr, NU, dinv, Y, LDY);
        trsm_lower_t<NU, NX + 1, NT>(g, Lr, NU, dinv, Y, LDY);  // Y = R^-1 [S | r]
    } else {
        trsm_lower<NU, 1, NT>(g, Lr, NU, dinv, Y + NX, LDY);
        trsm_lower_t<NU, 1, NT>(g, Lr, NU, dinv, Y + NX, LDY);  // y = R^-1 r
    }
    mm<NX, NX, NU, true, false, NT, false>(g, e + E::C, NX, Z, NX, Z, NX);  // C = Z^T Z
    mm<NX, 1, NU, false, false, NT, false>(g, e + E::b, 1, st + L::B, NU, Y + NX, LDY,
                                           st + L::c, 1, -1.f);            // b = c - B y
    if (has_S) {
        mm<NX, NX, NU, false, false, NT, false>(g, e + E::A, NX, st + L::B, NU, Y, LDY,
                                                st + L::A, NX, -1.f);
        mm<NX, NX, NU, true, false, NT, false>(g, e + E::P, NX, st + L::S, NX, Y, LDY,
                                               st + L::Q, NX, -1.f);
        mm<NX, 1, NU, true, false, NT, false>(g, e + E::p, 1, st + L::S, NX, Y + NX, LDY,
                                              st + L::q, 1, -1.f);
    } else {
        copy<NX, NX, false, NT, false>(g, e + E::A, NX, st + L::A, NX);
        copy<NX, NX, false, NT, false>(g, e + E::P, NX, st + L::Q, NX);
        for (int i = g.t; i < NX; i += NT) e[E::p + i] = st[L::q + i];
    }
    g.sync();
    return ok;
}

// ----------------------------------------------------------------- combines
// M^-1 [RHS] of a combine (Eq. combination_rule): the FP32 elimination, or,
// when m64 is set on a size that has it (n = 36, whose units of 128 threads
// hold one column of [M | A1 | C1 | b] each), the FP64 one (gj_solve_f64),
// its multiplier columns in the unit's shared tile buffer or else in the
// combine scratch at dscr (T, unused until M^-1 has been applied).
// (Out of line, so that its FP64 column registers do not weigh on the
// register allocation of the FP32 path around it.)
template <int NX, int NR, int NT>
__device__ __noinline__ bool m_solve_f64(const Grp<NT>& g, float* G, int ld, double* dbuf)
{
    return gj_solve_f64<NX, NR, NT>(g, G, ld, dbuf);
}

template <int NX, int NR, int NT>
__device__ __forceinline__ bool m_solve(const Grp<NT>& g, float* G, int ld, float* wsc,
                                        float* dscr, bool m64)
{
    if constexpr (NX == 36 && NX + NR <= NT) {
        if (m64) return m_solve_f64<NX, NR, NT>(g, G, ld, reinterpret_cast<double*>(g.tb ? g.tb : dscr));
    }
    // units with a factor buffer large enough for M (the split scan's CTAs at
    // n >= 96, the whole-body size's units): LU with partial pivoting of M in
    // shared memory, the right-hand sides solved in blocks there, instead of
    // the elimination in place in the work area
    if constexpr ((NX >= kSmemFactorRows || NX == 36) && NT >= SMEM_CB && NT % SMEM_CB == 0) {
        if (g.fb && g.fbn >= spd_smem_floats(NX)) return lu_solve_smem<NX, NR, NT>(g, G, ld, G + NX, ld, wsc);
    }
    return gj_solve<NX, NR, NT>(g, G, ld, wsc);
}

// out = e1 (x) e2 for two full elements (e1 earlier in time).  out must not
// alias e2; it may alias e1 on the one-warp path through M^-1 (every read of
// e1 there precedes the barrier before the first store to out, except the
// addends P1, p1, which each thread reads at the places it then writes).
template <int NX, int NT>
__device__ bool combine_full(const Grp<NT>& g, const float* e1, const float* e2, float* out,
                             float* scr, bool m64 = false)
{
    using E = ElemL<NX>;
    using S = CombL<NX>;
    if constexpr (WarpPath<NX, NX, NT>::inv) {
        // one warp: M^-1 by Gauss-Jordan on [M | I] (one column per lane),
        // then X_A = M^-1 A1, X_C = M^-1 C1, x_b = M^-1 (b1 - C1 p2) by products
        constexpr int LD = S::LDI;
        float* G = scr + S::GI;
        float* XA = scr + S::XA;
        float* XC = scr + S::XC;
        float* U = scr + S::UI;
        float* w = scr + S::wI;
        float* xb = scr + S::xb;
        float* vb = scr + S::vb;
        float* T = scr + S::GI;   // written once M^-1 is no longer read
        mm<NX, NX, NX, false, false, NT, false>(g, G, LD, e1 + E::C, NX, e2 + E::P, NX);
        fill<NX, NX, NT, false>(g, G + NX, LD, 0.f, 1.f);
        mm<NX, 1, NX, false, false, NT, false>(g, vb, 1, e1 + E::C, NX, e2 + E::p, 1, e1 + E::b, 1,
                                               -1.f);
        mm<NX, NX, NX, false, false, NT, false>(g, U, NX, e2 + E::P, NX, e1 + E::A, NX);
        mm<NX, 1, NX, false, false, NT, false>(g, w, 1, e2 + E::P, NX, e1 + E::b, 1, e2 + E::p, 1);
        g.sync();
        for (int i = g.t; i < NX; i += NT) G[i * LD + i] += 1.f;   // M = I + C1 P2
        g.sync();
        const bool ok = gj_warp<NX, NX>(g.t, G, LD, scr + S::WkI);
        const float* Mi = G + NX;
        mm<NX, NX, NX, false, false, NT, false>(g, XA, NX, Mi, LD, e1 + E::A, NX);
        mm<NX, NX, NX, false, false, NT, false>(g, XC, NX, Mi, LD, e1 + E::C, NX);
        mm<NX, 1, NX, false, false, NT, false>(g, xb, 1, Mi, LD, vb, 1);
        g.sync();
        mm<NX, NX, NX, false, false, NT, false>(g, out + E::A, NX, e2 + E::A, NX, XA, NX);
        mm<NX, 1, NX, false, false, NT, false>(g, out + E::b, 1, e2 + E::A, NX, xb, 1, e2 + E::b, 1);
        mm<NX, NX, NX, false, false, NT, false>(g, T, NX, e2 + E::A, NX, XC, NX);
        mm<NX, NX, NX, true, false, NT, false>(g, out + E::P, NX, XA, NX, U, NX, e1 + E::P, NX);
        mm<NX, 1, NX, true, false, NT, false>(g, out + E::p, 1, XA, NX, w, 1, e1 + E::p, 1);
        g.sync();
        mm<NX, NX, NX, false, true, NT>(g, out + E::C, NX, T, NX, e2 + E::A, NX, e2 + E::C, NX);
        symmetrize<NX, NT, false>(g, out + E::C, NX);
        symmetrize<NX, NT>(g, out + E::P, NX);
        return ok;
    }
    constexpr int LDG = S::LDG;
    float* G = scr + S::G;
    float* T = scr + S::T;
    float* U = scr + S::U;
    float* w = scr + S::w;
    // G = [C1 P2 | A1 | C1 | b1 - C1 p2];  U = P2 A1;  w = p2 + P2 b1
    mm<NX, NX, NX, false, false, NT, false>(g, G, LDG, e1 + E::C, NX, e2 + E::P, NX);
    copy<NX, NX, false, NT, false>(g, G + NX, LDG, e1 + E::A, NX);
    copy<NX, NX, false, NT, false>(g, G + 2 * NX, LDG, e1 + E::C, NX);
    mm<NX, 1, NX, false, false, NT, false>(g, G + 3 * NX, LDG, e1 + E::C, NX, e2 + E::p, 1,
                                           e1 + E::b, 1, -1.f);
    mm<NX, NX, NX, false, false, NT, false>(g, U, NX, e2 + E::P, NX, e1 + E::A, NX);
    mm<NX, 1, NX, false, false, NT, false>(g, w, 1, e2 + E::P, NX, e1 + E::b, 1, e2 + E::p, 1);
    g.sync();
    for (int i = g.t; i < NX; i += NT) G[i * LDG + i] += 1.f;   // M = I + C1 P2
    g.sync();
    const bool ok = m_solve<NX, 2 * NX + 1, NT>(g, G, LDG, scr + S::Wk, scr + S::T, m64);
    const float* XA = G + NX;       // M^-1 A1
    const float* XC = G + 2 * NX;   // M^-1 C1
    const float* xb = G + 3 * NX;   // M^-1 (b1 - C1 p2)
    mm<NX, NX, NX, false, false, NT, false>(g, out + E::A, NX, e2 + E::A, NX, XA, LDG);
    mm<NX, 1, NX, false, false, NT, false>(g, out + E::b, 1, e2 + E::A, NX, xb, LDG,
                                           e2 + E::b, 1);
    mm<NX, NX, NX, false, false, NT, false>(g, T, NX, e2 + E::A, NX, XC, LDG);
    mm<NX, NX, NX, true, false, NT, false>(g, out + E::P, NX, XA, LDG, U, NX, e1 + E::P, NX);
    mm<NX, 1, NX, true, false, NT, false>(g, out + E::p, 1, XA, LDG, w, 1, e1 + E::p, 1);
    g.sync();
    mm<NX, NX, NX, false, true, NT>(g, out + E::C, NX, T, NX, e2 + E::A, NX, e2 + E::C, NX);
    symmetrize<NX, NT, false>(g, out + E::C, NX);
    symmetrize<NX, NT>(g, out + E::P, NX);
    return ok;
}

// out(P, p) = e1 (x) V2 where V2 is a value function (A2 = C2 = b2 = 0):
// P = (M^-1 A1)^T P2 A1 + P1,  p = (M^-1 A1)^T (p2 + P2 b1) + p1.
template <int NX, int NT>
__device__ bool combine_vf(const Grp<NT>& g, const float* e1, const float* v2, float* out,
                           float* scr, bool m64 = false)
{
    using E = ElemL<NX>;
    using S = CombL<NX>;
    constexpr int LDG = 2 * NX;
    float* G = scr + S::G;
    float* U = scr + S::U;
    float* w = scr + S::w;
    mm<NX, NX, NX, false, false, NT, false>(g, G, LDG, e1 + E::C, NX, v2 + E::P, NX);
    copy<NX, NX, false, NT, false>(g, G + NX, LDG, e1 + E::A, NX);
    mm<NX, NX, NX, false, false, NT, false>(g, U, NX, v2 + E::P, NX, e1 + E::A, NX);
    mm<NX, 1, NX, false, false, NT, false>(g, w, 1, v2 + E::P, NX, e1 + E::b, 1, v2 + E::p, 1);
    g.sync();
    for (int i = g.t; i < NX; i += NT) G[i * LDG + i] += 1.f;
    g.sync();
    const bool ok = m_solve<NX, NX, NT>(g, G, LDG, scr + S::Wk, scr + S::T, m64);
    const float* XA = G + NX;
    mm<NX, NX, NX, true, false, NT, false>(g, out + E::P, NX, XA, LDG, U, NX, e1 + E::P, NX);
    mm<NX, 1, NX, true, false, NT, false>(g, out + E::p, 1, XA, LDG, w, 1, e1 + E::p, 1);
    g.sync();
    symmetrize<NX, NT>(g, out + E::P, NX);
    return ok;
}

// ------------------------------------------------------------ Riccati step
// Given V_{k+1} = (P', p') and stage k, evaluate Eq. (lqr):
//   G = R + B^T P' B,  H = S + B^T P' A,  h = B^T (p' + P' c) + r,
//   K = -G^-1 H,  k = -G^-1 h,
//   P = Q + A^T P' A + K^T H,  p = q + A^T (p' + P' c) + K^T h,
// with G^-1 [H | h] from one SPD elimination without pivoting (one warp,
// K^T [H | h] = -(G^-1 H)^T [H | h]) or, for wider systems, from the Cholesky
// factor G = L L^T: with [Z | z] = L^-1 [H | h], K^T H = -Z^T Z and
// K^T h = -Z^T z.  vin and vout hold value functions [P | p] (NX^2 + NX
// floats).  Writes P, p into vout, Abar = A + B K and bbar = B k + c into
// scr + RicL::Ab and scr + RicL::bb, and K, k, P, p, Abar, bbar to global
// memory at stage gs.
template <int NX, int NU, int NT, bool FAC = false>
__device__ bool riccati_step(const Grp<NT>& g, const float* st, const float* vin, float* vout,
                             float* scr, const KktArgs& a, int64_t gs, bool has_S)
{
    using L = StageL<NX, NU>;
    using S = RicL<NX, NU>;
    constexpr int LDY = NX + 1;
    float* PB = scr + S::PB;
    float* PA = scr + S::PA;
    float* w = scr + S::w;
    float* Gm = scr + S::G;
    float* dinv = scr + S::dinv;
    float* Y = scr + S::Y;
    float* Y2 = scr + S::Y2;
    const float* P1 = vin;
    const float* p1 = vin + NX * NX;
    float* P = vout;
    float* p = vout + NX * NX;
    mm<NX, NU, NX, false, false, NT, false>(g, PB, NU, P1, NX, st + L::B, NU);
    mm<NX, NX, NX, false, false, NT, false>(g, PA, NX, P1, NX, st + L::A, NX);
    mm<NX, 1, NX, false, false, NT, false>(g, w, 1, P1, NX, st + L::c, 1, p1, 1);
    g.sync();
    mm<NU, NU, NX, true, false, NT, false>(g, Gm, NU, st + L::B, NU, PB, NU, st + L::R, NU);
    mm<NU, NX, NX, true, false, NT, false>(g, Y, LDY, st + L::B, NU, PA, NX,
                                           has_S ? st + L::S : nullptr, NX);
    mm<NU, 1, NX, true, false, NT, false>(g, Y + NX, LDY, st + L::B, NU, w, 1, st + L::r, 1);
    // P = Q + A^T (P' A) ;  p = q + A^T w  (the K^T [H | h] terms follow)
    mm<NX, NX, NX, true, false, NT, false>(g, P, NX, st + L::A, NX, PA, NX, st + L::Q, NX);
    mm<NX, 1, NX, true, false, NT, false>(g, p, 1, st + L::A, NX, w, 1, st + L::q, 1);
    g.sync();
    // Y2 = G^-1 [H | h];  Yr = the factor paired with Y in K^T [H | h]:
    // G^-1 [H | h] itself (SPD elimination, Y untouched) or, after a Cholesky
    // factorisation G = L L^T, Y = L^-1 [H | h] paired with itself
    constexpr bool SPD = WarpPath<NX, NU, NT>::spd || WarpPath<NX, NU, NT>::spd_wide;
    bool ok;
    if constexpr (WarpPath<NX, NU, NT>::spd) {
        ok = spd_solve_warp<NU, NX + 1>(g.t, Gm, NU, Y, LDY, Y2, LDY, scr + S::Wk);
    } else if constexpr (WarpPath<NX, NU, NT>::spd_wide) {
        copy<NU, NX + 1, false, NT>(g, Y2, LDY, Y, LDY);
        bool done = false;
        if constexpr (FAC) {
            if (g.fb && g.fbn >= spd_smem_floats(NU)) {
                ok = spd_solve_smem<NU, NX + 1, NT>(g, Gm, NU, Y2, LDY, dinv);
                done = true;
            }
        }
        if (!done) ok = spd_solve_generic<NU, NX + 1, NT>(g, Gm, NU, Y2, LDY, dinv);
    } else {
        ok = chol<NU, NT>(g, Gm, NU, dinv, scr + S::Wk);
        trsm_lower<NU, NX + 1, NT>(g, Gm, NU, dinv, Y, LDY);           // [Z | z]
        copy<NU, NX + 1, false, NT>(g, Y2, LDY, Y, LDY);
        trsm_lower_t<NU, NX + 1, NT>(g, Gm, NU, dinv, Y2, LDY);        // G^-1 [H | h]
    }
    const float* Yr = SPD ? Y2 : Y;
    g.sync();
    // P += K^T H ;  p += K^T h
    mm<NX, NX, NU, true, false, NT, false>(g, P, NX, Y, LDY, Yr, LDY, P, NX, -1.f);
    mm<NX, 1, NU, true, false, NT, false>(g, p, 1, Y, LDY, Yr + NX, LDY, p, 1, -1.f);
    // K = -Y2[:, :NX], k = -Y2[:, NX];  Abar = A + B K;  bbar = B k + c
    float* Kg = a.K + gs * NU * NX;
    float* kg = a.k + gs * NU;
    if (NX % 4 == 0 && (reinterpret_cast<uintptr_t>(Kg) & 15) == 0) {
        for (int e = g.t; e < NU * NX / 4; e += NT) {
            const float* y = Y2 + ((4 * e) / NX) * LDY + (4 * e) % NX;
            reinterpret_cast<float4*>(Kg)[e] = make_float4(-y[0], -y[1], -y[2], -y[3]);
        }
    } else {
        for (int e = g.t; e < NU * NX; e += NT) Kg[e] = -Y2[(e / NX) * LDY + (e % NX)];
    }
    for (int i = g.t; i < NU; i += NT) kg[i] = -Y2[i * LDY + NX];
    float* Ab = scr + S::Ab;
    float* bb = scr + S::bb;
    mm<NX, NX, NU, false, false, NT, false>(g, Ab, NX, st + L::B, NU, Y2, LDY, st + L::A, NX, -1.f);
    mm<NX, 1, NU, false, false, NT, false>(g, bb, 1, st + L::B, NU, Y2 + NX, LDY, st + L::c, 1, -1.f);
    g.sync();
    symmetrize<NX, NT>(g, P, NX);
    store_out<NX * NX, NT>(g.t, a.P + gs * NX * NX, P);
    store_out<NX, NT>(g.t, a.p + gs * NX, p);
    store_out<NX * NX, NT>(g.t, a.Abar + gs * NX * NX, Ab);
    store_out<NX, NT>(g.t, a.bbar + gs * NX, bb);
    return ok;
}

// Terminal stage: V_N = (Q_N, q_N), K_N = 0, k_N = 0.
template <int NX, int NU, int NT>
__device__ void terminal_value(const Grp<NT>& g, const float* st, float* vout, const KktArgs& a,
                               int64_t gs)
{
    using L = StageL<NX, NU>;
    for (int e = g.t; e < NX * NX; e += NT) {
        vout[e] = st[L::Q + e];
        a.P[gs * NX * NX + e] = st[L::Q + e];
    }
    for (int i = g.t; i < NX; i += NT) {
        vout[NX * NX + i] = st[L::q + i];
        a.p[gs * NX + i] = st[L::q + i];
    }
    for (int e = g.t; e < NU * NX; e += NT) a.K[gs * NU * NX + e] = 0.f;
    for (int i = g.t; i < NU; i += NT) a.k[gs * NU + i] = 0.f;
    g.sync();
}

// Roll the trajectory of stages [k0, k1) forward from x (SMEM, length NX):
// dx_k = x, du_k = K_k x + k_k, dlam_k = P_k x + p_k, x <- Abar_k x + bbar_k.
// The per-stage operands are staged asynchronously, the next stage's while
// the current one is used (two buffers of RollL::SIZE floats at buf).
template <int NX, int NU>
struct RollL {
    static constexpr int K = 0, k = round4(NU * NX), P = round4(k + NU), p = round4(P + NX * NX),
                         Ab = round4(p + NX), bb = round4(Ab + NX * NX), SIZE = round4(bb + NX);
};

template <int NX, int NU, int NT>
__device__ __forceinline__ void roll_fetch(const Grp<NT>& g, float* b, const KktArgs& a, int64_t gs,
                                           bool terminal)
{
    using L = RollL<NX, NU>;
    stage_copy<NX * NX, NT, true>(g.t, b + L::P, a.P + gs * NX * NX);
    stage_copy<NX, NT, true>(g.t, b + L::p, a.p + gs * NX);
    if (!terminal) {
        stage_copy<NU * NX, NT, true>(g.t, b + L::K, a.K + gs * NU * NX);
        stage_copy<NU, NT, true>(g.t, b + L::k, a.k + gs * NU);
        stage_copy<NX * NX, NT, true>(g.t, b + L::Ab, a.Abar + gs * NX * NX);
        stage_copy<NX, NT, true>(g.t, b + L::bb, a.bbar + gs * NX);
    }
    cp_async_commit();
}

// Returns false on a thread that wrote a non-finite dx, du or dlam (a NaN or
// Inf anywhere in the inputs reaches these outputs).
template <int NX, int NU, int NT>
__device__ bool rollout_chunk(const Grp<NT>& g, float* x, float* xn, float* buf, const KktArgs& a,
                              int64_t off, int N, int k0, int k1)
{
    using L = RollL<NX, NU>;
    if (k0 >= k1) return true;
    bool fin = true;
    roll_fetch<NX, NU, NT>(g, buf, a, off + k0, k0 == N);
    for (int k = k0; k < k1; ++k) {
        const int64_t gs = off + k;
        float* cur = buf + ((k - k0) & 1) * L::SIZE;
        if (k + 1 < k1) {
            roll_fetch<NX, NU, NT>(g, buf + ((k + 1 - k0) & 1) * L::SIZE, a, gs + 1, k + 1 == N);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        g.sync();
        for (int i = g.t; i < NX; i += NT) {
            a.dx[gs * NX + i] = x[i];
            fin = fin && isfinite(x[i]);
        }
        mv<NX, NX, false, NT, false>(g, a.dlam + gs * NX, cur + L::P, NX, x, cur + L::p);
        if (k < N) {
            mv<NU, NX, false, NT, false>(g, a.du + gs * NU, cur + L::K, NX, x, cur + L::k);
            mv<NX, NX, false, NT, false>(g, xn, cur + L::Ab, NX, x, cur + L::bb);
            g.sync();
            for (int i = g.t; i < NX; i += NT) x[i] = xn[i];
            for (int i = g.t; i < NU; i += NT) fin = fin && isfinite(a.du[gs * NU + i]);
        } else {
            for (int i = g.t; i < NU; i += NT) a.du[gs * NU + i] = 0.f;
        }
        g.sync();
        for (int i = g.t; i < NX; i += NT) fin = fin && isfinite(a.dlam[gs * NX + i]);
    }
    return fin;
}

// ---------------------------------------------------------- chunk partition
// Chunk w of W over S = N+1 stages: every chunk gets one stage, the rest is
// shared in proportion to weights 10 (first and middle chunks) and 16 (the
// last chunk, whose value-function recursion runs while the middle chunks
// fold the costlier full combines).
__device__ __forceinline__ int chunk_start(int w, int W, int S)
{
    if (w >= W) return S;
    const int units = (W - 1) * 10 + 16;
    const int extra = S - W;
    return w + (int)(((int64_t)extra * (w * 10)) / units);
}

// ------------------------------------------------------------- scan kernel
template <int NX, int NU, int W>
struct ScanSmem {
    static constexpr int ELEM = ElemL<NX>::SIZE;
    static constexpr int STG = StageL<NX, NU>::SIZE;
    static constexpr int VF = round4(NX * NX + NX);   // a value function [P | p]
    // one-warp units fold their chunk in place (the combine through M^-1 reads
    // the earlier element completely before it overwrites it)
    static constexpr bool INPLACE = 2 * NX <= 32;
    // phase 1 (middle chunk): stage | build scratch, the combine's scratch
    // over both (the stage is dead by then), then elem (| tmpE)
    static constexpr int SB = STG + BuildL<NX, NU>::SIZE;
    static constexpr int ELEM_AT = round4(SB > CombL<NX>::SIZE ? SB : CombL<NX>::SIZE);
    static constexpr int P1 = ELEM_AT + (INPLACE ? 1 : 2) * ELEM;
    // phase 2: result | combine scratch
    static constexpr int P2 = 2 * ELEM + CombL<NX>::SIZE;
    // phase 1 (last chunk) / phase 3: stage | V0 | V1 | riccati scratch (the
    // chunk's closed-loop map is composed in its own slot)
    static constexpr int P3 = STG + 2 * VF + RicL<NX, NU>::SIZE;
    static constexpr int P4 = 2 * round4(NX) + 2 * RollL<NX, NU>::SIZE;
    // a chunk slot holds its aggregate element, later its map (Psi, psi)
    static constexpr int MAP = 2 * NX * NX + 2 * round4(NX);
    static constexpr int SLOT = round4(ELEM > MAP ? ELEM : MAP);
    static constexpr int PA_ = P1 > P2 ? P1 : P2;
    static constexpr int PB_ = P3 > P4 ? P3 : P4;
    static constexpr int PRIV = round4(PA_ > PB_ ? PA_ : PB_);
    static constexpr int SLOTS = W * SLOT;
    static constexpr int XS = W * round4(NX);
    static constexpr int TOTAL = SLOTS + W * PRIV + XS + 4;  // + status words
    static constexpr size_t BYTES = sizeof(float) * TOTAL;
    // phase 3 reads the boundary value function [P | p] (ends before ELEM) at
    // the start of the next chunk's private area while that chunk writes its
    // own v0 at STG: the two ranges must not overlap
    static_assert(ELEM <= STG, "boundary value function and v0 overlap");
};

// Tile buffers of the wide units (one TileBuf per unit), placed after a
// kernel's own dynamic shared memory (base bytes) when they fit.
template <int W, int UW>
struct UnitTiles {
    static constexpr size_t BYTES = UW > 1 ? (size_t)W * TileBuf::FLOATS * sizeof(float) : 0;
    __host__ __device__ static constexpr size_t at(size_t base) { return (base + 15) & ~(size_t)15; }
    __host__ __device__ static constexpr bool fit(size_t base)
    {
        return BYTES > 0 && at(base) + BYTES <= kSmemCta;
    }
    __host__ __device__ static constexpr size_t total(size_t base)
    {
        return fit(base) ? at(base) + BYTES : base;
    }
};

// Factor buffers of the wide units (shared-memory SPD solves), placed after
// the tile buffers for kernels whose work areas live in global memory, when
// they fit.  For systems of 96 rows or more (smaller augmented matrices stay
// in L1 through the elimination in place, and the buffer would take that L1
// away from the products), and for the whole-body size (n, m) = (36, 24),
// whose 4-warp units spent their time in the barriers and global-memory
// reads of the in-place eliminations.  The buffer holds max(NX, NU) rows:
// the SPD systems have NU, the combines' M has NX.
template <int NU, int W, int UW, int NX = NU>
struct UnitFactor {
    static constexpr int ROWS = NX > NU ? NX : NU;
    static constexpr bool ON = UW > 1 && (NU >= kSmemFactorRows || (NX == 36 && NU == 24));
    static constexpr int FLOATS = ON ? spd_smem_floats(ROWS) : 0;
    static constexpr size_t BYTES = (size_t)W * FLOATS * sizeof(float);
    __host__ __device__ static constexpr size_t at(size_t base) { return (base + 15) & ~(size_t)15; }
    __host__ __device__ static constexpr bool fit(size_t base)
    {
        return BYTES > 0 && at(base) + BYTES <= kSmemCta;
    }
    __host__ __device__ static constexpr size_t total(size_t base)
    {
        return fit(base) ? at(base) + BYTES : base;
    }
};

// Configurations whose products go through the tensor cores: one chunk
// owned by a 256-thread unit (the whole CTA) with a factor buffer that can
// stage the products.
template <int NX, int NU, int W, int UW>
struct UseTc {
    static constexpr int R = NX > NU ? NX : NU;
    static constexpr bool value = W == 1 && UW == 8 && UnitFactor<NU, W, UW>::FLOATS >= tc_stage_floats(R, R);
    static constexpr uint32_t cols = (uint32_t)tc_cols(R);
};

// Barrier of the W CTAs that share one instance in the split scan (one CTA
// per horizon chunk, launched cooperatively so that all of them are
// resident): every CTA adds one to the instance's counter and waits until it
// reaches `target` (phase number x W).  The writes of all threads of a CTA
// before the barrier are published by thread 0's fence before its arrival,
// and the fence after the wait orders the reads that follow.  The wait is
// bounded (2 s by the global timer): a barrier that does not complete sets
// `late` (thread 0's) and lets the CTA go on, so that the kernel always ends;
// once late, the CTA still arrives at later barriers but waits at none, so
// that a failed instance costs one timeout, not one per phase.  skip_arrive
// (a test switch) leaves this CTA's arrival out, so that the others' wait
// runs out with nothing in flight.
__device__ __forceinline__ void split_barrier(unsigned* cnt, unsigned target, int& late,
                                              bool skip_arrive = false)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (!skip_arrive) atomicAdd(cnt, 1u);
        const uint64_t t0 = globaltimer_ns();
        while (!late && *(volatile unsigned*)cnt < target) {
            if (globaltimer_ns() - t0 > 2000000000ull) {
                late = 1;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
}

// The scan solve of one instance by the CTA (all threads must call it).
// src provides the LQ stages; s_inst points to this instance's dx_0 (global
// or shared memory).  Returns the instance status (uniform over the CTA).
//
// The horizon is split into W chunks, each owned by a unit of UW warps
// (NT = 32 UW threads: one warp for small states, several for large ones,
// synchronised by a named barrier per unit).
//
// SPLIT: the chunks run on separate CTAs (chunk = blockIdx.x, one unit per
// CTA, launched cooperatively), smem is the instance's work area in global
// memory, tiles / factors / tc belong to this CTA's single unit, and the
// barriers between phases are split_barrier on the instance's counter sbar.
template <int NX, int NU, int W, int UW, class Src, bool SPLIT = false>
__device__ int scan_solve(const Src& src, const KktArgs& a, int N, int64_t off,
                          const float* s_inst, float* smem, float* tiles = nullptr,
                          float* factors = nullptr, TcCtx* tc = nullptr, unsigned* sbar = nullptr)
{
    using SM = ScanSmem<NX, NU, W>;
    using E = ElemL<NX>;
    constexpr int NT = 32 * UW;
    constexpr int WU = SPLIT ? 1 : W;      // units per CTA
    const int warp = SPLIT ? (int)blockIdx.x : (int)(threadIdx.x / NT);   // the chunk
    const int unit = SPLIT ? 0 : warp;     // the unit within this CTA
    using UF = UnitFactor<NU, WU, UW, NX>;
    // factor buffers exist for this configuration (the caller passes them
    // whenever they fit); the shared-memory solves are compiled only then
    constexpr bool FAC = UF::FLOATS > 0 && UF::BYTES + UnitTiles<WU, UW>::BYTES + 1024 <= kSmemCta;
    const Grp<NT> g{(int)(threadIdx.x % NT), 1 + unit,
                    tiles ? tiles + unit * TileBuf::FLOATS : nullptr,
                    factors ? factors + (size_t)unit * UF::FLOATS : nullptr, factors ? UF::FLOATS : 0,
                    tc};
    // barrier between phases: the CTA, or the instance's CTAs in split mode
    int late = 0;             // thread 0: a split barrier that ran out
    unsigned sb_phase = 0;
    auto phase_sync = [&]() {
        if constexpr (SPLIT) {
            ++sb_phase;
            const bool skip = (a.dbg & PDILQR_DEBUG_SPLIT_SKIP_ARRIVE) && warp == 0 && sb_phase == 1;
            split_barrier(sbar, sb_phase * (unsigned)gridDim.x, late, skip);
        } else {
            __syncthreads();
        }
    };
    const int S = N + 1;
    const int Weff = W < S ? W : S;
    const bool has_S = src.has_S();

    float* slots = smem;                               // [W][ELEM]
    float* priv = smem + SM::SLOTS + warp * SM::PRIV;  // this warp's private area
    float* xs = smem + SM::SLOTS + W * SM::PRIV;       // [W][NX] chunk start states
    int* st_word = reinterpret_cast<int*>(xs + SM::XS);
    if (threadIdx.x == 0) st_word[0] = ST_OK;
    phase_sync();

    const int k0 = chunk_start(warp, Weff, S);
    const int k1 = chunk_start(warp + 1, Weff, S);
    const bool active = warp < Weff;
    const bool last = warp == Weff - 1;
    int bad = ST_OK;

    // ---- phase 1
    float* stg = priv;
    if (active && !last && warp > 0) {
        // fold e_{k0} (x) ... (x) e_{k1-1} into slots[warp]: the stage and the
        // build scratch first, the combine scratch over both
        static_assert(!SM::INPLACE || WarpPath<NX, NX, NT>::inv, "in-place fold needs the M^-1 combine");
        float* bscr = priv + SM::STG;
        float* cscr = priv;
        float* elem = priv + SM::ELEM_AT;
        float* acc = slots + warp * SM::SLOT;
        float* other = SM::INPLACE ? acc : elem + SM::ELEM;
        for (int k = k0; k < k1; ++k) {
            src.template load<NX, NU, NT>(g, stg, off + k, false);
            src.template keep<NX, NU, NT>(g, stg, off + k);
            if (k == k0) {
                if (!build_element<NX, NU, NT, FAC>(g, stg, acc, bscr, has_S, false)) bad = ST_NOT_SPD;
            } else {
                if (!build_element<NX, NU, NT, FAC>(g, stg, elem, bscr, has_S, false)) bad = ST_NOT_SPD;
                if (!combine_full<NX, NT>(g, acc, elem, other, cscr, a.m64)) bad = ST_SINGULAR;
                float* t = acc; acc = other; other = t;
            }
        }
        if (acc != slots + warp * SM::SLOT) copy<E::SIZE, 1, false, NT>(g, slots + warp * SM::SLOT, 1, acc, 1);
    } else if (Src::kKeeps && active && !last && warp == 0) {
        // the first chunk has no fold to do: prepare its stages for the sweep
        // (for sources that linearise on the fly this moves the work off the
        // sweep's critical path)
        for (int k = k0; k < k1; ++k) {
            src.template load<NX, NU, NT>(g, stg, off + k, false);
            src.template keep<NX, NU, NT>(g, stg, off + k);
        }
    } else if (active && last) {
        // value-function recursion of the last chunk from the terminal cost
        float* v0 = priv + SM::STG;
        float* v1 = v0 + SM::VF;
        float* scr = v1 + SM::VF;
        for (int k = k1 - 1; k >= k0; --k) {
            src.template load<NX, NU, NT>(g, stg, off + k, k == N);
            if (k == N) {
                terminal_value<NX, NU, NT>(g, stg, v0, a, off + k);
            } else {
                if (!riccati_step<NX, NU, NT, FAC>(g, stg, v0, v1, scr, a, off + k, has_S)) bad = ST_NOT_SPD;
                float* t = v0; v0 = v1; v1 = t;
            }
        }
        copy<NX * NX + NX, 1, false, NT>(g, slots + warp * SM::SLOT + E::P, 1, v0, 1);
    }
    phase_sync();

    // ---- phase 2: suffix scan over the chunk aggregates, items 0..J-1 of
    // chunks 1..Weff-1 (the last is a value function).  The levels alternate
    // between two copies of the items, the chunk slots (A) and the result
    // buffers at the start of the chunks' private areas (B), so that a level
    // ends with one barrier; item j ends up holding the value function at the
    // start of chunk j + 1.  Items that no longer combine are value functions
    // and carry their P, p across.
    const int J = Weff - 1;
    float* const bufA = slots;                 // item i at bufA + (i + 1) SLOT
    float* const bufB = smem + SM::SLOTS;      // item i at bufB + (i + 1) PRIV
    bool in_b = false;                         // the copy holding the items
    {
        const int j = warp - 1;
        float* scr = priv + SM::ELEM;          // after this chunk's own B item
        for (int d = 1; d < J; d <<= 1) {
            const float* src = in_b ? bufB : bufA;
            float* dst = in_b ? bufA : bufB;
            const int ss = in_b ? SM::PRIV : SM::SLOT;
            const int ds = in_b ? SM::SLOT : SM::PRIV;
            if (j >= 0 && j < J) {
                const float* e1 = src + (j + 1) * ss;
                float* out = dst + (j + 1) * ds;
                if (j + d < J) {
                    const bool vf = (j + 2 * d - 1 >= J - 1);
                    const float* e2 = src + (j + 1 + d) * ss;
                    const bool ok = vf ? combine_vf<NX, NT>(g, e1, e2, out, scr, a.m64)
                                       : combine_full<NX, NT>(g, e1, e2, out, scr + SM::ELEM, a.m64);
                    if (!ok) bad = ST_SINGULAR;
                } else {
                    copy<NX * NX + NX, 1, false, NT>(g, out + E::P, 1, e1 + E::P, 1);
                }
            }
            phase_sync();
            in_b = !in_b;
        }
    }

    // ---- phase 3: Riccati sweep of chunks 0..Weff-2 from their boundary
    // value functions, composing the chunk's closed-loop affine map.
    // the chunk's map (Psi, psi) is composed in its own slot once the chunk
    // before has taken its boundary value function from there
    float* psiA = slots + warp * SM::SLOT;
    float* psiB = psiA + NX * NX;
    float* psiv = psiB + NX * NX;
    float* psitmp = psiv + round4(NX);
    float* v0 = priv + SM::STG;
    float* v1 = v0 + SM::VF;
    if (active && !last) {
        const float* vb = in_b ? bufB + (warp + 1) * SM::PRIV : bufA + (warp + 1) * SM::SLOT;
        copy<NX * NX + NX, 1, false, NT, false>(g, v0, 1, vb + E::P, 1);
    }
    phase_sync();
    if (active && !last) {
        float* scr = v1 + SM::VF;
        fill<NX, NX, NT, false>(g, psiA, NX, 0.f, 1.f);
        for (int i = g.t; i < NX; i += NT) psiv[i] = 0.f;
        g.sync();
        for (int k = k1 - 1; k >= k0; --k) {
            const int64_t gs = off + k;
            src.template reload<NX, NU, NT>(g, stg, gs);   // kept in phase 1
            if (!riccati_step<NX, NU, NT, FAC>(g, stg, v0, v1, scr, a, gs, has_S)) bad = ST_NOT_SPD;
            float* t = v0; v0 = v1; v1 = t;
            __threadfence_block();
            g.sync();
            // psi <- Psi bbar_k + psi ;  Psi <- Psi Abar_k
            // (Abar_k, bbar_k as the Riccati step left them in its scratch)
            mm<NX, 1, NX, false, false, NT, false>(g, psitmp, 1, psiA, NX, scr + RicL<NX, NU>::bb, 1, psiv, 1);
            mm<NX, NX, NX, false, false, NT, false>(g, psiB, NX, psiA, NX, scr + RicL<NX, NU>::Ab, NX);
            g.sync();
            for (int i = g.t; i < NX; i += NT) psiv[i] = psitmp[i];
            float* t2 = psiA; psiA = psiB; psiB = t2;
            g.sync();
        }
        // publish Psi, psi at the fixed place in this chunk's slot
        if (psiA != slots + warp * SM::SLOT) copy<NX * NX, 1, false, NT>(g, slots + warp * SM::SLOT, 1, psiA, 1);
    }
    if (bad != ST_OK && g.t == 0) atomicMax(st_word, bad);
    phase_sync();

    // ---- phase 4: trajectory scan.  Chunk start states from dx_0 through the
    // chunk maps, then every chunk rolls out dx, du, dlam.
    if (warp == 0) {
        float* x = xs;
        for (int i = g.t; i < NX; i += NT) x[i] = s_inst[i];
        g.sync();
        for (int w = 0; w + 1 < Weff; ++w) {
            const float* Psi = slots + w * SM::SLOT;
            const float* psv = Psi + 2 * NX * NX;
            mv<NX, NX, false, NT>(g, xs + (w + 1) * round4(NX), Psi, NX, xs + w * round4(NX), psv);
        }
    }
    phase_sync();
    if (active) {
        float* x = priv;                 // reuse the private area
        float* xn = priv + round4(NX);
        float* rb = priv + 2 * round4(NX);
        for (int i = g.t; i < NX; i += NT) x[i] = xs[warp * round4(NX) + i];
        g.sync();
        if (!rollout_chunk<NX, NU, NT>(g, x, xn, rb, a, off, N, k0, k1)) atomicMax(st_word, ST_NONFINITE);
    }
    phase_sync();
    if constexpr (SPLIT) {
        // every CTA's timeouts (barrier or tensor-core wait) reach the status
        if (threadIdx.x == 0 && (late || (tc && tc->failed))) atomicMax(st_word, ST_TIMEOUT);
        phase_sync();
    }
    int status = st_word[0];
    // a tensor-core product whose bounded wait ran out (uniform over the CTA)
    if (tc && tc->failed) status = ST_TIMEOUT;
    phase_sync();
    return status;
}

// Warps per unit (one horizon chunk): one warp for small states, a group of
// warps for large ones.
template <int NX>
struct UnitWarps {
    static constexpr int value = NX <= 24 ? 1 : (NX <= 36 ? 4 : 8);
};

// CTAs per SM the register budget is sized for: 16 warps per SM with up to
// 128 registers per thread.  Holding the one-robot kernels to fewer registers
// for more warps per SM made them slower (80 registers and 24 warps: the
// 8-chunk batch 86 ms against 72 ms; 96 registers and 20 one-warp CTAs: the
// sequential recursion 2 % faster on the batch, 5.6 % slower on one instance).
template <int WARPS>
struct MinBlocks {
    static constexpr int value = WARPS >= 16 ? 1 : (WARPS >= 8 ? 2 : (WARPS >= 4 ? 4 : 16));
};

template <int NX, int NU, int W, int UW>
__global__ void __launch_bounds__(W * 32 * UW, MinBlocks<W * UW>::value)
    kkt_scan_kernel(const __grid_constant__ KktArgs a)
{
    extern __shared__ __align__(16) float smem[];
    using TL = UnitTiles<W, UW>;
    const int inst = a.order ? a.order[blockIdx.x] : blockIdx.x;
    if (inst >= a.count) return;
    const LqSource src(a);
    float* work = a.gws ? a.gws + (int64_t)blockIdx.x * ScanSmem<NX, NU, W>::TOTAL : smem;
    using UF = UnitFactor<NU, W, UW, NX>;
    const size_t base = a.gws ? 0 : ScanSmem<NX, NU, W>::BYTES;
    float* tiles = TL::fit(base) ? smem + TL::at(base) / sizeof(float) : nullptr;
    const size_t fbase = TL::total(base);
    float* factors = (a.gws && UF::fit(fbase)) ? smem + UF::at(fbase) / sizeof(float) : nullptr;
    TcCtx* tc = nullptr;
    if constexpr (UseTc<NX, NU, W, UW>::value) {
        __shared__ TcCtx tcx;
        if (factors) {
            tc_setup(&tcx, UseTc<NX, NU, W, UW>::cols, (a.dbg & PDILQR_DEBUG_TC_SKIP_ISSUE) != 0);
            tc = &tcx;
        }
    }
    const int st = scan_solve<NX, NU, W, UW>(src, a, a.N[inst], a.off[inst],
                                             a.s + (int64_t)inst * NX, work, tiles, factors, tc);
    if (tc) tc_teardown(tc);
    if (threadIdx.x == 0) a.status[inst] = st;
}


// The split scan (Sec. II-D over several SMs): one CTA per horizon chunk
// (blockIdx.x) and one grid row per instance (blockIdx.y, longest first),
// launched cooperatively so that the W CTAs of an instance are resident
// together and meet at the bounded phase barriers (a.sbar[row], zeroed
// before the launch).  Each CTA is one unit of UW warps with its own tile
// buffer, factor buffer and, where the one-chunk kernels have them,
// tensor-core products; the instance's chunk aggregates and work areas live
// in the global workspace (ScanSmem<NX, NU, W>::TOTAL floats per instance).
template <int NX, int NU, int W, int UW>
__global__ void __launch_bounds__(32 * UW, 1) kkt_scan_split_kernel(const __grid_constant__ KktArgs a)
{
    extern __shared__ __align__(16) float smem[];
    using TL = UnitTiles<1, UW>;
    using UF = UnitFactor<NU, 1, UW>;
    if ((int)blockIdx.y >= a.count) return;   // a whole grid row: no barrier waits on it
    const int inst = a.order ? a.order[blockIdx.y] : (int)blockIdx.y;
    const LqSource src(a);
    float* work = a.gws + (int64_t)blockIdx.y * ScanSmem<NX, NU, W>::TOTAL;
    float* tiles = TL::fit(0) ? smem + TL::at(0) / sizeof(float) : nullptr;
    const size_t fbase = TL::total(0);
    float* factors = UF::fit(fbase) ? smem + UF::at(fbase) / sizeof(float) : nullptr;
    TcCtx* tc = nullptr;
    if constexpr (UseTc<NX, NU, 1, UW>::value) {
        __shared__ TcCtx tcx;
        if (factors) {
            tc_setup(&tcx, UseTc<NX, NU, 1, UW>::cols, (a.dbg & PDILQR_DEBUG_TC_SKIP_ISSUE) != 0);
            tc = &tcx;
        }
    }
    const int st = scan_solve<NX, NU, W, UW, LqSource, true>(src, a, a.N[inst], a.off[inst],
                                                             a.s + (int64_t)inst * NX, work, tiles,
                                                             factors, tc, a.sbar + blockIdx.y);
    if (tc) tc_teardown(tc);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.status[inst] = st;
}

// Scan solve for the allocation-free entry point: the batch tables come from
// the caller, so every instance's slot range is checked against the scratch
// capacity (limit stage slots) before any access; an instance that does not
// fit is reported as invalid and skipped.
template <int NX, int NU, int W>
__global__ void __launch_bounds__(W * 32, MinBlocks<W>::value)
    kkt_scan_checked_kernel(const __grid_constant__ KktArgs a, int64_t limit)
{
    extern __shared__ __align__(16) float smem[];
    const int inst = blockIdx.x;
    if (inst >= a.count) return;
    const int N = a.N[inst];
    const int64_t off = a.off[inst];
    if (N < 1 || N > 4096 || off < 0 || off + N + 1 > limit) {
        if (threadIdx.x == 0) a.status[inst] = ST_INVALID_ARG;
        return;
    }
    const LqSource src(a);
    const int st = scan_solve<NX, NU, W, 1>(src, a, N, off, a.s + (int64_t)inst * NX, smem);
    if (threadIdx.x == 0) a.status[inst] = st;
}

// --------------------------------------------------------- Riccati kernel
template <int NX, int NU>
struct RicSmem {
    static constexpr int ELEM = ElemL<NX>::SIZE;
    static constexpr int STG = StageL<NX, NU>::SIZE;
    static constexpr int VF = round4(NX * NX + NX);
    static constexpr int TOTAL = STG + 2 * VF + RicL<NX, NU>::SIZE + 2 * round4(NX) +
                                 2 * RollL<NX, NU>::SIZE;
    static constexpr size_t BYTES = sizeof(float) * TOTAL;
};

// One warp per instance; blockDim.x = 32 * warps-per-block.
template <int NX, int NU>
__global__ void __launch_bounds__(128) riccati_kernel(const __grid_constant__ KktArgs a)
{
    using SM = RicSmem<NX, NU>;
    extern __shared__ __align__(16) float smem[];
    const int warp = threadIdx.x >> 5;
    const int slot = blockIdx.x * (blockDim.x >> 5) + warp;
    if (slot >= a.count) return;
    const int inst = a.order ? a.order[slot] : slot;
    const Grp<32> g{(int)(threadIdx.x & 31), 0};
    float* base = smem + warp * SM::TOTAL;
    float* stg = base;
    float* v0 = base + SM::STG;
    float* v1 = v0 + SM::VF;
    float* scr = v1 + SM::VF;
    float* x = scr + RicL<NX, NU>::SIZE;
    float* xn = x + round4(NX);
    float* rb = xn + round4(NX);
    const int N = a.N[inst];
    const int64_t off = a.off[inst];
    int bad = ST_OK;
    load_stage<NX, NU, 32>(g, stg, a, off + N, true);
    terminal_value<NX, NU, 32>(g, stg, v0, a, off + N);
    for (int k = N - 1; k >= 0; --k) {
        load_stage<NX, NU, 32>(g, stg, a, off + k, false);
        if (!riccati_step<NX, NU, 32>(g, stg, v0, v1, scr, a, off + k, a.S != nullptr))
            bad = ST_NOT_SPD;
        float* t = v0; v0 = v1; v1 = t;
    }
    __threadfence_block();
    for (int i = g.t; i < NX; i += 32) x[i] = a.s[(int64_t)inst * NX + i];
    g.sync();
    const bool fin = rollout_chunk<NX, NU, 32>(g, x, xn, rb, a, off, N, 0, N + 1);
    if (__any_sync(0xffffffffu, !fin)) bad = ST_NONFINITE;
    if (g.t == 0) a.status[inst] = bad;
}

}  // namespace pdl
