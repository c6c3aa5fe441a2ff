// scan_rows.cuh -- the parallel associative scan of Sec. II-D with one matrix
// row per lane: each horizon chunk is a 16-lane half-warp, lane r holding
// row r of the blocks it forms, so that the element build (Eq.
// initialization), the combines of Eq. (combination_rule) and the Riccati
// sweeps run on the register-resident row operations of sqp_rows.cuh.
//
// Elements are kept in shared memory in the ElemL layout (A, C, b, P, p,
// row-major); a value function uses P, p only.  Combine (e1 earlier in time):
//   M = I + C1 P2,
//   A = A2 M^-1 A1,            b = A2 M^-1 (b1 - C1 p2) + b2,
//   C = A2 M^-1 C1 A2^T + C2,  P = (M^-1 A1)^T P2 A1 + P1,
//   p = (M^-1 A1)^T (p2 + P2 b1) + p1.
#pragma once

#include "sqp_rows.cuh"

namespace pdl {

// The element build, the combines and (through riccati_rows_ool) the
// Riccati step are kept out of line in the scan kernel:
// inlined at every call site they made the scan kernel's body too large for
// the instruction cache (instruction-fetch stalls were the second largest
// stall reason), and out of line the single-instance SQP iteration is about
// 15 % faster.

// The Riccati step of the scan kernel, out of line (the sequential kernel
// inlines it: there it is the only large operation, and out of line it cost
// that kernel 2.5x per step).
template <int N>
__device__ __noinline__ bool riccati_rows_ool(const Grp<16>& g, const float* st, float* scr,
                                              const KktArgs& a, int64_t gs, float* abar_sm)
{
    return riccati_rows<N>(g, st, scr, a, gs, false, abar_sm);
}

// ------------------------------------------------------ row eliminations
// G^-1 Y for an SPD N x N matrix G by Gauss-Jordan elimination without
// pivoting, rows per lane (lane r < N: row r of G in gr, of Y in yr): step k
// takes row k from lane k by shuffles and every other row subtracts its
// multiple; at the end each row is divided by its pivot.  For an SPD matrix
// the pivots are the diagonal of its L D L^T factorisation, so "every pivot
// positive and finite" is the SPD test.  Lanes >= N must hold zeros.  On exit
// yr is row r of G^-1 Y.  Returns the test (uniform over the half).
template <int N, int NR>
__device__ __forceinline__ bool gj_rows_spd(const Grp<16>& g, float (&gr)[N], float (&yr)[NR])
{
    const int r = g.t;
    bool ok = true;
    float dr = 1.f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const float pk = __shfl_sync(g.mask, gr[k], k, 16);
        ok = ok && (pk > 0.f) && isfinite(pk);
        if (r == k) dr = pk;
        const float f = (r < N && r != k) ? gr[k] * rcp_approx(pk) : 0.f;
#pragma unroll
        for (int j = k + 1; j < N; ++j) gr[j] = fmaf(-f, __shfl_sync(g.mask, gr[j], k, 16), gr[j]);
#pragma unroll
        for (int j = 0; j < NR; ++j) yr[j] = fmaf(-f, __shfl_sync(g.mask, yr[j], k, 16), yr[j]);
    }
    const float idr = rcp_approx(dr);
#pragma unroll
    for (int j = 0; j < NR; ++j) yr[j] *= idr;
    return ok;
}

// M^-1 Y for a general N x N matrix M by Gauss-Jordan elimination with
// partial pivoting, rows per lane (lane r < N: row r of M in mr, of Y in yr).
// The rows are not exchanged: step k picks the unused row whose column-k
// entry is largest in magnitude (a shuffle reduction, ties to the lower
// lane), and every other row subtracts its multiple of that row; the lane
// that pivoted column k ends holding unknown k.  On exit yr is row `unk` of
// M^-1 Y (lanes >= N: unk = -1).  Returns false (uniformly) if a pivot is
// below 1e-30 in magnitude or not finite.
template <int N, int NR>
__device__ __forceinline__ bool gj_rows_piv(const Grp<16>& g, float (&mr)[N], float (&yr)[NR], int& unk)
{
    const int r = g.t;
    bool used = r >= N;
    bool ok = true;
    float dr = 1.f;
    unk = -1;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        float v = used ? -1.f : fabsf(mr[k]);
        int idx = r;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(g.mask, v, o, 16);
            const int oi = __shfl_xor_sync(g.mask, idx, o, 16);
            if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
        }
        const int p = idx;
        const float pk = __shfl_sync(g.mask, mr[k], p, 16);
        ok = ok && (fabsf(pk) > 1e-30f) && isfinite(pk);
        if (r == p) { used = true; unk = k; dr = pk; }
        const float f = (r < N && r != p) ? mr[k] * rcp_approx(pk) : 0.f;
#pragma unroll
        for (int j = k + 1; j < N; ++j) mr[j] = fmaf(-f, __shfl_sync(g.mask, mr[j], p, 16), mr[j]);
#pragma unroll
        for (int j = 0; j < NR; ++j) yr[j] = fmaf(-f, __shfl_sync(g.mask, yr[j], p, 16), yr[j]);
    }
    const float idr = rcp_approx(dr);
#pragma unroll
    for (int j = 0; j < NR; ++j) yr[j] *= idr;
    return ok;
}

// row r of X (N-wide rows, row-major at X) times the rows of Y: out[j] =
// sum_l X[r][l] Y[l][j] + (D ? D[j] : 0), with X's row in registers (xr)
template <int N>
__device__ __forceinline__ void row_times(const float (&xr)[N], const float* Y, float (&out)[N])
{
#pragma unroll
    for (int l = 0; l < N; ++l) {
        float yl[N];
        ld_row(yl, Y + l * N);
#pragma unroll
        for (int j = 0; j < N; ++j) out[j] = fmaf(xr[l], yl[j], out[j]);
    }
}

// M <- (M + M^T) / 2 for a row-major N x N matrix in shared memory, rows per
// lane (every read precedes the barrier before the first write).  Ends with
// a barrier of the half.
template <int N>
__device__ __forceinline__ void symmetrize_rows(const Grp<16>& g, float* M)
{
    const int r = g.t;
    float mr[N];
    if (r < N) {
        ld_row(mr, M + r * N);
#pragma unroll
        for (int j = 0; j < N; ++j) mr[j] = 0.5f * (mr[j] + M[j * N + r]);
    }
    g.sync();
    if (r < N) st_row(M + r * N, mr);
    g.sync();
}

// ------------------------------------------------------------ element build
// Scratch of the row element build and combines, per chunk (floats, every
// block 16-byte aligned).
template <int N>
struct RowElemScr {
    static constexpr int X = 0, y = X + N * N, U = round4(y + N), w = U + N * N,
                         XA = round4(w + N), XC = XA + N * N, xb = XC + N * N,
                         T = round4(xb + N), SIZE = round4(T + N * N);
};

// e_k = (A, C, b, P, p) = (A - B R^-1 S, B R^-1 B^T, c - B R^-1 r, Q - S^T R^-1 S,
// q - S^T R^-1 r) of Eq. (initialization), here with S = 0, from the stage
// st (StageL layout) into e (ElemL layout), rows per lane: R^-1 [B^T | r] by
// the SPD elimination (lane r: row r of R and column r of B), then C = B X
// and b = c - B y from the rows of X = R^-1 B^T; C is symmetrised.  Returns
// false if R is not SPD.  Ends with a barrier of the half.
template <int N>
__device__ __noinline__ bool build_element_rows(const Grp<16>& g, const float* st, float* e, float* scr)
{
    using L = StageL<N, N>;
    using E = ElemL<N>;
    using S = RowElemScr<N>;
    const int r = g.t;
    const bool row = r < N;
    float rr[N], xr[N + 1];
#pragma unroll
    for (int j = 0; j < N; ++j) { rr[j] = 0.f; xr[j] = 0.f; }
    xr[N] = 0.f;
    if (row) {
        ld_row(rr, st + L::R + r * N);
#pragma unroll
        for (int j = 0; j < N; ++j) xr[j] = st[L::B + j * N + r];   // column r of B
        xr[N] = st[L::r + r];
    }
    const bool ok = gj_rows_spd<N, N + 1>(g, rr, xr);
    if (row) {
        float xs[N];
#pragma unroll
        for (int j = 0; j < N; ++j) xs[j] = xr[j];
        st_row(scr + S::X + r * N, xs);
        scr[S::y + r] = xr[N];
    }
    g.sync();
    if (row) {
        float br[N], cr[N], ar[N], qr[N];
        ld_row(br, st + L::B + r * N);
#pragma unroll
        for (int j = 0; j < N; ++j) cr[j] = 0.f;
        row_times(br, scr + S::X, cr);
        float bv = st[L::c + r];
#pragma unroll
        for (int l = 0; l < N; ++l) bv = fmaf(-br[l], scr[S::y + l], bv);
        st_row(e + E::C + r * N, cr);
        ld_row(ar, st + L::A + r * N);
        st_row(e + E::A + r * N, ar);
        ld_row(qr, st + L::Q + r * N);
        st_row(e + E::P + r * N, qr);
        e[E::b + r] = bv;
        e[E::p + r] = st[L::q + r];
    }
    g.sync();
    symmetrize_rows<N>(g, e + E::C);
    return ok;
}

// ----------------------------------------------------------------- combines
// out = e1 (x) e2 for two full elements (e1 earlier in time), rows per lane;
// out must not alias e1 or e2.  M = I + C1 P2 is eliminated with partial
// pivoting together with [A1 | C1 | b1 - C1 p2]; the solution rows go to the
// scratch at their unknowns' positions, then lane r forms row r of
// A = A2 X_A, T = A2 X_C, C = T A2^T + C2, P = X_A^T (P2 A1) + P1 and
// b_r, p_r.  C and P are symmetrised.  Returns false if M is singular.
template <int N>
__device__ __noinline__ bool combine_full_rows(const Grp<16>& g, const float* e1, const float* e2, float* out,
                                  float* scr)
{
    using E = ElemL<N>;
    using S = RowElemScr<N>;
    const int r = g.t;
    const bool row = r < N;
    float mr[N], yr[2 * N + 1];
#pragma unroll
    for (int j = 0; j < N; ++j) mr[j] = 0.f;
#pragma unroll
    for (int j = 0; j < 2 * N + 1; ++j) yr[j] = 0.f;
    if (row) {
        float c1[N], a1[N], p2r[N], u[N];
        ld_row(c1, e1 + E::C + r * N);
        row_times(c1, e2 + E::P, mr);                 // C1 P2
#pragma unroll
        for (int j = 0; j < N; ++j) mr[j] += (j == r) ? 1.f : 0.f;
        ld_row(a1, e1 + E::A + r * N);
        float bv = e1[E::b + r];
#pragma unroll
        for (int l = 0; l < N; ++l) bv = fmaf(-c1[l], e2[E::p + l], bv);
#pragma unroll
        for (int j = 0; j < N; ++j) { yr[j] = a1[j]; yr[N + j] = c1[j]; }
        yr[2 * N] = bv;
        ld_row(p2r, e2 + E::P + r * N);
#pragma unroll
        for (int j = 0; j < N; ++j) u[j] = 0.f;
        row_times(p2r, e1 + E::A, u);                 // U = P2 A1
        float wr = e2[E::p + r];
#pragma unroll
        for (int l = 0; l < N; ++l) wr = fmaf(p2r[l], e1[E::b + l], wr);   // w = p2 + P2 b1
        st_row(scr + S::U + r * N, u);
        scr[S::w + r] = wr;
    }
    int unk;
    const bool ok = gj_rows_piv<N, 2 * N + 1>(g, mr, yr, unk);
    if (unk >= 0) {
        float xa[N], xc[N];
#pragma unroll
        for (int j = 0; j < N; ++j) { xa[j] = yr[j]; xc[j] = yr[N + j]; }
        st_row(scr + S::XA + unk * N, xa);
        st_row(scr + S::XC + unk * N, xc);
        scr[S::xb + unk] = yr[2 * N];
    }
    g.sync();
    if (row) {
        float a2[N], ar[N], tr[N], pr[N], cr[N];
        ld_row(a2, e2 + E::A + r * N);
#pragma unroll
        for (int j = 0; j < N; ++j) { ar[j] = 0.f; tr[j] = 0.f; }
        row_times(a2, scr + S::XA, ar);               // A2 X_A
        row_times(a2, scr + S::XC, tr);               // A2 X_C
        float bv = e2[E::b + r];
#pragma unroll
        for (int l = 0; l < N; ++l) bv = fmaf(a2[l], scr[S::xb + l], bv);
        ld_row(pr, e1 + E::P + r * N);
        float pv = e1[E::p + r];
#pragma unroll
        for (int l = 0; l < N; ++l) {                  // X_A^T U + P1, X_A^T w + p1
            const float xlr = scr[S::XA + l * N + r];
            float ul[N];
            ld_row(ul, scr + S::U + l * N);
#pragma unroll
            for (int j = 0; j < N; ++j) pr[j] = fmaf(xlr, ul[j], pr[j]);
            pv = fmaf(xlr, scr[S::w + l], pv);
        }
        ld_row(cr, e2 + E::C + r * N);
#pragma unroll
        for (int j = 0; j < N; ++j) {                  // T A2^T + C2
            float a2j[N];
            ld_row(a2j, e2 + E::A + j * N);
#pragma unroll
            for (int l = 0; l < N; ++l) cr[j] = fmaf(tr[l], a2j[l], cr[j]);
        }
        st_row(out + E::A + r * N, ar);
        st_row(out + E::C + r * N, cr);
        st_row(out + E::P + r * N, pr);
        out[E::b + r] = bv;
        out[E::p + r] = pv;
    }
    g.sync();
    symmetrize_rows<N>(g, out + E::C);
    symmetrize_rows<N>(g, out + E::P);
    return ok;
}

// out (P, p) = e1 (x) V2 for a value function V2 (A2 = C2 = b2 = 0):
// P = (M^-1 A1)^T P2 A1 + P1, p = (M^-1 A1)^T (p2 + P2 b1) + p1, rows per
// lane; out must not alias e1 or v2.  P is symmetrised.
template <int N>
__device__ __noinline__ bool combine_vf_rows(const Grp<16>& g, const float* e1, const float* v2, float* out,
                                float* scr)
{
    using E = ElemL<N>;
    using S = RowElemScr<N>;
    const int r = g.t;
    const bool row = r < N;
    float mr[N], yr[N];
#pragma unroll
    for (int j = 0; j < N; ++j) { mr[j] = 0.f; yr[j] = 0.f; }
    if (row) {
        float c1[N], p2r[N], u[N];
        ld_row(c1, e1 + E::C + r * N);
        row_times(c1, v2 + E::P, mr);
#pragma unroll
        for (int j = 0; j < N; ++j) mr[j] += (j == r) ? 1.f : 0.f;
        ld_row(yr, e1 + E::A + r * N);
        ld_row(p2r, v2 + E::P + r * N);
#pragma unroll
        for (int j = 0; j < N; ++j) u[j] = 0.f;
        row_times(p2r, e1 + E::A, u);
        float wr = v2[E::p + r];
#pragma unroll
        for (int l = 0; l < N; ++l) wr = fmaf(p2r[l], e1[E::b + l], wr);
        st_row(scr + S::U + r * N, u);
        scr[S::w + r] = wr;
    }
    int unk;
    const bool ok = gj_rows_piv<N, N>(g, mr, yr, unk);
    if (unk >= 0) st_row(scr + S::XA + unk * N, yr);
    g.sync();
    if (row) {
        float pr[N];
        ld_row(pr, e1 + E::P + r * N);
        float pv = e1[E::p + r];
#pragma unroll
        for (int l = 0; l < N; ++l) {
            const float xlr = scr[S::XA + l * N + r];
            float ul[N];
            ld_row(ul, scr + S::U + l * N);
#pragma unroll
            for (int j = 0; j < N; ++j) pr[j] = fmaf(xlr, ul[j], pr[j]);
            pv = fmaf(xlr, scr[S::w + l], pv);
        }
        st_row(out + E::P + r * N, pr);
        out[E::p + r] = pv;
    }
    g.sync();
    symmetrize_rows<N>(g, out + E::P);
    return ok;
}

// ------------------------------------------------------------- the kernel
// Shared memory of one horizon chunk (floats, 16-byte aligned blocks).
template <int NX>
struct ScanRowsChunk {
    using L = StageL<NX, NX>;
    using E = ElemL<NX>;
    static constexpr int INF = round4(SrbdSource::in_floats<NX, NX>());
    static constexpr int ST = 0;                      // linearised stage
    static constexpr int INB = round4(ST + L::SIZE);  // two stage-input buffers
    static constexpr int AG = INB + 2 * INF;          // two element buffers: the fold's
                                                      // accumulator, the suffix scan's two
                                                      // copies of the item, the chunk map
    static constexpr int UN = AG + 2 * E::SIZE;       // scratch of the phase
    // phases 1-2: element scratch, a built element
    static constexpr int ESCR = UN, ELEM = UN + round4(RowElemScr<NX>::SIZE);
    // phase 1 (last chunk) and phase 3: Riccati scratch, the step's Abar rows and bbar
    static constexpr int RSCR = UN, ABS = UN + round4(RowRicL<NX>::SIZE);
    static constexpr int UN_END = (ELEM + E::SIZE) > (ABS + NX * NX + NX) ? (ELEM + E::SIZE)
                                                                           : (ABS + NX * NX + NX);
    static constexpr int XS = round4(UN_END);         // the chunk's start state / rollout state
    static constexpr int SIZE = round4(XS + 16);
    static_assert(L::SIZE >= 16 * 46 && RowElemScr<NX>::SIZE >= 16 * 24, "merit buffers fit");
};

template <int NX, int W>
struct ScanRowsSmem {
    using C = ScanRowsChunk<NX>;
    static constexpr int MERH = W * C::SIZE;          // per-half merit sums, W x 26 doubles
    static constexpr int MER = MERH + W * 2 * 26;     // merit of the instance, 26 doubles
    static constexpr int CTL = MER + 2 * 26;          // step size, flags, status word
    static constexpr int TOTAL = round4(CTL + 8);
    static constexpr size_t BYTES = sizeof(float) * TOTAL;
};

// The fused SQP of Sec. II-B..II-E with the LQ KKT system solved by the
// parallel scan of Sec. II-D for the single-robot SRBD model (n = m = 12),
// one instance per CTA of W half-warps.  Chunk c (half-warp c) owns stages
// [chunk_start(c), chunk_start(c + 1)) of the N + 1 (the partition of
// kkt_scan.cuh).  Per iteration:
//   phase 1  every chunk but the last linearises its stages (inputs fetched
//            one stage ahead) and keeps them for phase 3; the middle chunks
//            fold their elements e_k0 (x) ... (x) e_{k1-1}; the last chunk
//            runs the value-function recursion from the terminal cost;
//   phase 2  a Hillis-Steele suffix scan over the chunk aggregates gives the
//            value function at every chunk boundary;
//   phase 3  every chunk but the last runs the Riccati step (Eq. lqr) over
//            its stages from its boundary value function, composing its
//            closed-loop map (Psi, psi);
//   phase 4  the chunks' start states follow from dx_0 through the maps,
//            then every chunk rolls out dx, du, dlam;
// then the line search (all halves split the stages of the merit) and the
// update, as in sqp_rows_kernel.
template <int NX, int W>
__global__ void __launch_bounds__(16 * W, 1) sqp_scan_rows_kernel(const __grid_constant__ SqpArgs a)
{
    using C = ScanRowsChunk<NX>;
    using SM = ScanRowsSmem<NX, W>;
    using E = ElemL<NX>;
    using L = StageL<NX, NX>;
    using RS = RowRicL<NX>;
    constexpr int NU = NX;
    extern __shared__ __align__(16) float smem[];
    const int inst = a.ka.order ? a.ka.order[blockIdx.x] : blockIdx.x;
    if (inst >= a.ka.count) return;
    const int c = threadIdx.x >> 4;
    Grp<16> g{(int)(threadIdx.x & 15), 0};
    g.mask = 0xffffu << (16 * (c & 1));
    const int r = g.t;
    const bool row = r < NX;
    float* my = smem + c * C::SIZE;
    float* st = my + C::ST;
    float* inb = my + C::INB;
    float* ag = my + C::AG;
    float* escr = my + C::ESCR;
    float* elem = my + C::ELEM;
    float* rscr = my + C::RSCR;
    float* abs_ = my + C::ABS;
    float* xsc = my + C::XS;
    double* merh = reinterpret_cast<double*>(smem + SM::MERH);
    double* mer = reinterpret_cast<double*>(smem + SM::MER);
    float* alpha_sh = smem + SM::CTL;
    int* ctl = reinterpret_cast<int*>(smem + SM::CTL + 1);   // [0] stop, [1] full step, [2] status

    const KktArgs& ka = a.ka;
    const int N = ka.N[inst];
    const int64_t off = ka.off[inst];
    const int nrob = a.md.nrob;
    const SrbdSource src{a.md, a.x, a.u, a.lam, a.xref, a.uref, a.contact, nrob, a.lqcache};
    const float* xh = a.x0hat + (int64_t)inst * NX;
    float* x = a.x + off * NX;
    float* u = a.u + off * NU;
    float* lam = a.lam + off * NX;
    float* dx = ka.dx + off * NX;
    float* du = ka.du + off * NU;
    float* dl = ka.dlam + off * NX;
    const float* xr = a.xref + off * NX;
    const float* ur = a.uref + off * NU;
    const uint8_t* ct = a.contact + off * 4 * nrob;
    const int S = N + 1;
    const int Weff = W < S ? W : S;
    const int k0 = chunk_start(c, Weff, S), k1 = chunk_start(c + 1, Weff, S);
    const bool active = c < Weff, last = c == Weff - 1;
    auto item = [&](int j, bool b) { return smem + (j + 1) * C::SIZE + C::AG + (b ? E::SIZE : 0); };

    int status = ST_OK, iters = 0;
    for (int it = 0; it < a.max_iters; ++it) {
        if (threadIdx.x == 0) ctl[2] = ST_OK;
        __syncthreads();
        int bad = ST_OK;
        // ---- phase 1
        if (active && !last) {
            src.template fetch<NX, NU, 16>(g, inb + (k0 & 1) * C::INF, off + k0, false);
            int cur = 0;
            for (int k = k0; k < k1; ++k) {
                g.sync();
                if (k + 1 < k1) {
                    src.template fetch<NX, NU, 16>(g, inb + ((k + 1) & 1) * C::INF, off + k + 1, false);
                    src.template linearize<NX, NU, 16, 1>(g, st, inb + (k & 1) * C::INF, false);
                } else {
                    src.template linearize<NX, NU, 16, 0>(g, st, inb + (k & 1) * C::INF, false);
                }
                src.template keep<NX, NU, 16>(g, st, off + k);
                if (c > 0) {
                    if (k == k0) {
                        if (!build_element_rows<NX>(g, st, ag, escr)) bad = ST_NOT_SPD;
                    } else {
                        if (!build_element_rows<NX>(g, st, elem, escr)) bad = ST_NOT_SPD;
                        if (!combine_full_rows<NX>(g, ag + cur * E::SIZE, elem, ag + (1 - cur) * E::SIZE, escr))
                            bad = ST_SINGULAR;
                        cur ^= 1;
                    }
                }
            }
            if (c > 0 && cur) {
                for (int e = g.t; e < E::SIZE / 4; e += 16)
                    reinterpret_cast<float4*>(ag)[e] = reinterpret_cast<const float4*>(ag + E::SIZE)[e];
                g.sync();
            }
        } else if (active && last) {
            // value-function recursion from the terminal cost over stages N .. k0
            src.template fetch<NX, NU, 16>(g, inb + (N & 1) * C::INF, off + N, true);
            if (N - 1 >= k0) {
                src.template fetch<NX, NU, 16>(g, inb + ((N - 1) & 1) * C::INF, off + N - 1, false);
                src.template linearize<NX, NU, 16, 1>(g, st, inb + (N & 1) * C::INF, true);
            } else {
                src.template linearize<NX, NU, 16, 0>(g, st, inb + (N & 1) * C::INF, true);
            }
            if (row) {
                float PN[NX];
                ld_row(PN, st + L::Q + r * NX);
                const float pN = st[L::q + r];
                st_row(rscr + RS::V + r * NX, PN);
                rscr[RS::vp + r] = pN;
                st_row(ka.P + (off + N) * NX * NX + r * NX, PN);
                ka.p[(off + N) * NX + r] = pN;
            }
            for (int k = N - 1; k >= k0; --k) {
                g.sync();
                if (k - 1 >= k0) {
                    src.template fetch<NX, NU, 16>(g, inb + ((k - 1) & 1) * C::INF, off + k - 1, false);
                    src.template linearize<NX, NU, 16, 1>(g, st, inb + (k & 1) * C::INF, false);
                } else {
                    src.template linearize<NX, NU, 16, 0>(g, st, inb + (k & 1) * C::INF, false);
                }
                if (!riccati_rows_ool<NX>(g, st, rscr, ka, off + k, nullptr)) bad = ST_NOT_SPD;
            }
            g.sync();
            for (int e = g.t; e < NX * NX + NX; e += 16) ag[E::P + e] = rscr[RS::V + e];
            g.sync();
        }
        if (bad != ST_OK && g.t == 0) atomicMax(&ctl[2], bad);
        __syncthreads();
        // ---- phase 2: suffix scan over the aggregates of chunks 1 .. Weff-1
        // (item j of chunk j + 1; the last is a value function).  Two copies
        // of the items alternate, so a level ends with one barrier; items
        // that no longer combine are value functions and carry P, p across.
        const int J = Weff - 1;
        bool in_b = false;
        for (int d = 1; d < J; d <<= 1) {
            const int j = c - 1;
            if (j >= 0 && j < J) {
                const float* e1 = item(j, in_b);
                float* out = item(j, !in_b);
                if (j + d < J) {
                    const bool vf = (j + 2 * d - 1 >= J - 1);
                    const float* e2 = item(j + d, in_b);
                    const bool ok = vf ? combine_vf_rows<NX>(g, e1, e2, out, escr)
                                       : combine_full_rows<NX>(g, e1, e2, out, escr);
                    if (!ok && g.t == 0) atomicMax(&ctl[2], (int)ST_SINGULAR);
                } else {
                    for (int e = g.t; e < NX * NX + NX; e += 16) out[E::P + e] = e1[E::P + e];
                }
            }
            __syncthreads();
            in_b = !in_b;
        }
        // ---- phase 3: Riccati sweeps of chunks 0 .. Weff-2 from their boundary
        // value functions (item c), composing the chunk map Psi = Abar_{k1-1}
        // ... Abar_{k0}, psi (row r of Psi in registers)
        if (active && !last) {
            const float* vb = item(c, in_b);
            for (int e = g.t; e < NX * NX + NX; e += 16) rscr[RS::V + e] = vb[E::P + e];
        }
        __syncthreads();   // every boundary value function taken: the slots take the maps
        if (active && !last) {
            float Psi[NX], psv = 0.f;
#pragma unroll
            for (int j = 0; j < NX; ++j) Psi[j] = (j == r) ? 1.f : 0.f;
            bad = ST_OK;
            for (int k = k1 - 1; k >= k0; --k) {
                g.sync();
                src.template reload<NX, NU, 16>(g, st, off + k);
                if (!riccati_rows_ool<NX>(g, st, rscr, ka, off + k, abs_)) bad = ST_NOT_SPD;
                g.sync();
                if (row) {
                    // psi <- Psi bbar_k + psi ;  Psi <- Psi Abar_k
                    float np[NX];
#pragma unroll
                    for (int j = 0; j < NX; ++j) np[j] = 0.f;
#pragma unroll
                    for (int l = 0; l < NX; ++l) psv = fmaf(Psi[l], abs_[NX * NX + l], psv);
                    row_times(Psi, abs_, np);
#pragma unroll
                    for (int j = 0; j < NX; ++j) Psi[j] = np[j];
                }
            }
            if (row) {
                st_row(ag + r * NX, Psi);
                ag[NX * NX + r] = psv;
            }
            if (bad != ST_OK && g.t == 0) atomicMax(&ctl[2], bad);
        }
        __syncthreads();
        // ---- phase 4: chunk start states from dx_0 through the maps, then
        // every chunk rolls out its stages
        if (c == 0) {
            float xv = row ? xh[r] - x[r] : 0.f;
            if (row) xsc[r] = xv;
            for (int w = 0; w + 1 < Weff; ++w) {
                const float* Pm = smem + w * C::SIZE + C::AG;
                float* xw = smem + w * C::SIZE + C::XS;
                float* xn = smem + (w + 1) * C::SIZE + C::XS;
                g.sync();
                if (row) {
                    float pr[NX], xl[NX];
                    ld_row(pr, Pm + r * NX);
                    ld_row(xl, xw);
                    float v = Pm[NX * NX + r];
#pragma unroll
                    for (int j = 0; j < NX; ++j) v = fmaf(pr[j], xl[j], v);
                    xn[r] = v;
                }
            }
        }
        __syncthreads();
        if (active) {
            const float xv0 = row ? xsc[r] : 0.f;
            g.sync();
            const bool fin = rollout_rows<NX>(g, ka, off, N, k0, k1, xv0, xsc);
            if (__any_sync(g.mask, !fin) && g.t == 0) atomicMax(&ctl[2], (int)ST_NONFINITE);
        }
        __threadfence_block();
        __syncthreads();
        if (ctl[2] != ST_OK) {
            status = ctl[2];
            break;
        }
        iters = it + 1;
        // ---- line search (Sec. II-E): every half takes stages 16 c + lane,
        // + 16 W, ...; the full step first, the other nine only if it is rejected
        merit_rows<0, 0>(g, a.md, x, u, dx, du, xr, ur, ct, xh, N, st, escr, merh + 26 * c, 16 * c, 16 * W);
        __syncthreads();
        if (threadIdx.x < 26) {
            const int s = threadIdx.x;
            if (s < 3 || s == 3 || s == 13) {
                double v = 0.0;
                for (int h = 0; h < W; ++h) v += merh[26 * h + s];
                mer[s] = v;
            } else if (s == 23 || s == 25) {
                double v = 0.0;
                for (int h = 0; h < W; ++h) v = fmax(v, merh[26 * h + s]);
                mer[s] = v;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (it == 0) mer[24] = (double)a.theta_frac * fmax(1.0, mer[1]);
            const bool full = a.alpha_replay ? a.alpha_replay[(int64_t)inst * a.max_iters + it] == 1.f
                                             : filter_ok(mer[1], mer[2], mer[24], 1.0, mer[3], mer[13], a.c_armijo);
            ctl[1] = full ? 1 : 0;
        }
        __syncthreads();
        if (!ctl[1]) {
            merit_rows_rest(g, a.md, x, u, dx, du, xr, ur, ct, xh, N, st, escr, merh + 26 * c, 16 * c, 16 * W);
            __syncthreads();
            if (threadIdx.x < 23 && ((threadIdx.x >= 4 && threadIdx.x <= 12) || threadIdx.x >= 14)) {
                double v = 0.0;
                for (int h = 0; h < W; ++h) v += merh[26 * h + threadIdx.x];
                mer[threadIdx.x] = v;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double th0 = mer[1], dphi = mer[2];
            const double thmax = mer[24];
            float alpha = 0.f;
            double th_new = INFINITY;
            if (a.alpha_replay) {
                alpha = a.alpha_replay[(int64_t)inst * a.max_iters + it];
                for (int t = 0; t < 10; ++t)
                    if (alpha == ldexpf(1.f, -t) && (t == 0 || !ctl[1])) th_new = mer[13 + t];
            } else {
                for (int t = 0; t < (ctl[1] ? 1 : 10); ++t) {
                    const double at = ldexp(1.0, -t);
                    if (filter_ok(th0, dphi, thmax, at, mer[3 + t], mer[13 + t], a.c_armijo)) {
                        alpha = (float)at;
                        th_new = mer[13 + t];
                        break;
                    }
                }
            }
            const double floor_th = (double)(N + 1) * sqrt((double)NX) * 0x1p-23 * fmax(1.0, mer[25]);
            const bool at_floor = alpha == 0.f && th0 <= floor_th && !a.alpha_replay;
            alpha_sh[0] = at_floor ? -1.f : alpha;
            ctl[0] = (at_floor || (mer[23] < (double)a.tol_step && th_new < (double)a.tol_theta)) ? 1 : 0;
            if (a.alpha) a.alpha[(int64_t)inst * a.max_iters + it] = alpha;
        }
        __syncthreads();
        const float alpha = alpha_sh[0];
        if (alpha == 0.f) {
            status = ST_LINESEARCH;
            break;
        }
        if (alpha < 0.f) break;   // converged at the precision floor
        // ---- Eq. (linear_rollout): x += a dx, u += a du, lam += a dlam
        {
            float4* x4 = reinterpret_cast<float4*>(x);
            float4* l4 = reinterpret_cast<float4*>(lam);
            const float4* dx4 = reinterpret_cast<const float4*>(dx);
            const float4* dl4 = reinterpret_cast<const float4*>(dl);
            for (int e = threadIdx.x; e < (N + 1) * NX / 4; e += blockDim.x) {
                float4 v = x4[e], d = dx4[e];
                v.x += alpha * d.x; v.y += alpha * d.y; v.z += alpha * d.z; v.w += alpha * d.w;
                x4[e] = v;
                v = l4[e]; d = dl4[e];
                v.x += alpha * d.x; v.y += alpha * d.y; v.z += alpha * d.z; v.w += alpha * d.w;
                l4[e] = v;
            }
            float4* u4 = reinterpret_cast<float4*>(u);
            const float4* du4 = reinterpret_cast<const float4*>(du);
            for (int e = threadIdx.x; e < N * NU / 4; e += blockDim.x) {
                float4 v = u4[e], d = du4[e];
                v.x += alpha * d.x; v.y += alpha * d.y; v.z += alpha * d.z; v.w += alpha * d.w;
                u4[e] = v;
            }
        }
        __threadfence_block();
        __syncthreads();
        if (ctl[0]) break;
    }
    if (a.J || a.theta) {
        // merit at the returned iterate (only the current-point sums are read)
        merit_rows<0, 0>(g, a.md, x, u, dx, du, xr, ur, ct, xh, N, st, escr, merh + 26 * c, 16 * c, 16 * W);
        __syncthreads();
        if (threadIdx.x < 2) {
            double v = 0.0;
            for (int h = 0; h < W; ++h) v += merh[26 * h + threadIdx.x];
            mer[threadIdx.x] = v;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.iters[inst] = iters;
        a.status[inst] = status;
        if (a.J) a.J[inst] = mer[0];
        if (a.theta) a.theta[inst] = mer[1];
        if (a.alpha)
            for (int t = iters; t < a.max_iters; ++t) a.alpha[(int64_t)inst * a.max_iters + t] = 0.f;
    }
}

}  // namespace pdl
