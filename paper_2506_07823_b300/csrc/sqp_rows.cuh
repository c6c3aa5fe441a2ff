// sqp_rows.cuh -- the fused SQP of Sec. II-B..II-E with the LQ KKT system
// solved by the sequential Riccati recursion of Sec. II-C, one matrix row per
// lane: the batched solver for small states (n = m <= 16).
//
// Two instances share a warp, one per 16-lane half.  Lane r of a half holds
// row r of the value function P' and of every block the Riccati step forms
// (P'A, P'B, [G | H | h], the new P, Abar) in registers; the rows a lane
// needs from other lanes (rows of A, B, P'A, P'B, H, G^-1 H) are read from
// shared memory as 128-bit broadcasts, and the pivot rows of the elimination
// come by shuffles.  A
// 12 x 12 product is then 144 register FMAs per lane with 36 broadcast
// loads, and each issued instruction serves both instances of the warp.
// The stage data come from the SRBD linearisation (srbd.cuh), run by the
// same half.
#pragma once

#include "sqp.cuh"

namespace pdl {

// ------------------------------------------------------------ row helpers
template <int N>
__device__ __forceinline__ void ld_row(float (&v)[N], const float* p)
{
    static_assert(N % 4 == 0, "rows of whole float4");
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
        const float4 t = reinterpret_cast<const float4*>(p)[q];
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
    }
}

template <int N>
__device__ __forceinline__ void st_row(float* p, const float (&v)[N], float sgn = 1.f)
{
#pragma unroll
    for (int q = 0; q < N / 4; ++q)
        reinterpret_cast<float4*>(p)[q] =
            make_float4(sgn * v[4 * q], sgn * v[4 * q + 1], sgn * v[4 * q + 2], sgn * v[4 * q + 3]);
}

// Scratch of one row-per-lane Riccati step (floats; every block 16-byte
// aligned).  PA and PB hold the rows of P'A and P'B; once G, H and h are
// formed they are dead and hold the rows of G^-1 H (Y, over PA) and of H
// (over PB).  Pt: rows of P before symmetrisation; V, vp: the value function
// carried from step to step.
template <int N>
struct RowRicL {
    static constexpr int PA = 0, PB = PA + N * N, w = PB + N * N, hv = round4(w + N),
                         yv = round4(hv + N), Pt = round4(yv + N), V = Pt + N * N, vp = V + N * N,
                         SIZE = round4(vp + N);
    static constexpr int Y = PA, H = PB;
};

// One step of Eq. (lqr) for n = m = N by the 16 lanes of a half-warp:
//   G = R + B^T P' B,  H = S + B^T P' A,  h = r + B^T (p' + P' c),
//   K = -G^-1 H,  k = -G^-1 h,
//   P = Q + A^T P' A - H^T G^-1 H,  p = q + A^T (p' + P' c) - H^T G^-1 h,
//   Abar = A + B K,  bbar = c + B k.
// The value function V' = (P', p') lives in the scratch (rows at V, p' at
// vp) on entry and is replaced by the symmetrised (P, p) on exit, so that no
// register holds it between steps.  G^-1 [H | h] is formed by Gauss-Jordan
// elimination without pivoting on the rows [G | H | h] (lane r: row r): for
// an SPD G the pivots are the diagonal of its L D L^T factorisation, so
// "every pivot positive and finite" is the SPD test.  Rows of K, k, P, p,
// Abar, bbar are written to global memory at stage slot gs (Abar, bbar also
// to abar_sm when given: N rows, then N floats).  Returns false (uniformly
// over the half) if G is not SPD.
//
// lam1 (optional, n floats): the costate lam_{k+1} when the stage's q and r
// leave out their terms A^T lam_{k+1} and B^T lam_{k+1} (srbd_lin_rows12).
// Both enter the step only through A^T w and B^T w with w = p' + P'c, so
// adding lam_{k+1} to w adds them exactly where they belong.
template <int N>
__device__ bool riccati_rows(const Grp<16>& g, const float* st, float* scr, const KktArgs& a,
                             int64_t gs, bool has_S, float* abar_sm = nullptr,
                             const float* lam1 = nullptr)
{
    using L = StageL<N, N>;
    using S = RowRicL<N>;
    static_assert(N <= 16 && N % 4 == 0, "one row per lane of a half-warp");
    const int r = g.t;
    const bool row = r < N;
    float* PA = scr + S::PA;
    float* PB = scr + S::PB;
    float* w = scr + S::w;
    // (a) row r of P'A, P'B and w_r = (P'c + p')_r
    if (row) {
        float pa[N], pb[N];
#pragma unroll
        for (int j = 0; j < N; ++j) { pa[j] = 0.f; pb[j] = 0.f; }
        float wr = scr[S::vp + r];
        if (lam1) wr += lam1[r];
        // blocks of four rows l (the loop over blocks is not unrolled: a
        // smaller body keeps the two warps of a scheduler in the
        // instruction cache)
#pragma unroll 1
        for (int q = 0; q < N / 4; ++q) {
            const float4 p4 = reinterpret_cast<const float4*>(scr + S::V + r * N)[q];
            const float4 c4 = reinterpret_cast<const float4*>(st + L::c)[q];
            const float pq[4] = {p4.x, p4.y, p4.z, p4.w}, cq[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int l = 4 * q + i;
                float al[N], bl[N];
                ld_row(al, st + L::A + l * N);
                ld_row(bl, st + L::B + l * N);
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    pa[j] = fmaf(pq[i], al[j], pa[j]);
                    pb[j] = fmaf(pq[i], bl[j], pb[j]);
                }
                wr = fmaf(pq[i], cq[i], wr);
            }
        }
        st_row(PA + r * N, pa);
        st_row(PB + r * N, pb);
        w[r] = wr;
    }
    g.sync();
    // (b) rows of G, H, P and h_r, p_r: column r of B and A against the rows
    // of P'B, P'A and w
    float gr[N], hr[N], pn[N], hs = 0.f, ps = 0.f;
#pragma unroll
    for (int j = 0; j < N; ++j) { gr[j] = 0.f; hr[j] = 0.f; pn[j] = 0.f; }
    if (row) {
        ld_row(gr, st + L::R + r * N);
        ld_row(pn, st + L::Q + r * N);
        if (has_S) ld_row(hr, st + L::S + r * N);
        hs = st[L::r + r];
        ps = st[L::q + r];
        // two passes over the rows (G, h from P'B; H, P, p from P'A) keep
        // fewer accumulators live
#pragma unroll 4
        for (int l = 0; l < N; ++l) {
            const float blr = st[L::B + l * N + r];
            float pbl[N];
            ld_row(pbl, PB + l * N);
#pragma unroll
            for (int j = 0; j < N; ++j) gr[j] = fmaf(blr, pbl[j], gr[j]);
            hs = fmaf(blr, w[l], hs);
        }
#pragma unroll 4
        for (int l = 0; l < N; ++l) {
            const float blr = st[L::B + l * N + r], alr = st[L::A + l * N + r];
            float pal[N];
            ld_row(pal, PA + l * N);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                hr[j] = fmaf(blr, pal[j], hr[j]);
                pn[j] = fmaf(alr, pal[j], pn[j]);
            }
            ps = fmaf(alr, w[l], ps);
        }
    }
    g.sync();   // P'A, P'B and w are dead: their areas take H and Y
    float* H = scr + S::H;
    float* hv = scr + S::hv;
    if (row) {
        st_row(H + r * N, hr);
        hv[r] = hs;
    }
    // (c) G^-1 [H | h] by Gauss-Jordan elimination without pivoting, row r
    // per lane; at step k every other row subtracts its multiple of row k,
    // whose entries come from lane k by shuffles (no shared-memory round
    // trip or barrier); the pivot row is not normalised.  Column k of G is
    // not needed after step k, so every step shifts the row's remaining
    // columns of G left by one: the pivot column is always gr[0], and the
    // loop over k needs no unrolling (a small body for the instruction
    // cache, at the price of updating the dead columns too).
    bool ok = true;
    float dr = 1.f;
#pragma unroll 3
    for (int k = 0; k < N; ++k) {
        const float pk = __shfl_sync(g.mask, gr[0], k, 16);
        ok = ok && (pk > 0.f) && isfinite(pk);
        if (r == k) dr = pk;
        const float f = (row && r != k) ? gr[0] * rcp_approx(pk) : 0.f;
#pragma unroll
        for (int j = 1; j < N; ++j) gr[j - 1] = fmaf(-f, __shfl_sync(g.mask, gr[j], k, 16), gr[j]);
        gr[N - 1] = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) hr[j] = fmaf(-f, __shfl_sync(g.mask, hr[j], k, 16), hr[j]);
        hs = fmaf(-f, __shfl_sync(g.mask, hs, k, 16), hs);
    }
    // (d) Y = G^-1 H, y = G^-1 h (row r divided by its pivot); K = -Y, k = -y
    float* Y = scr + S::Y;
    float* yv = scr + S::yv;
    if (row) {
        const float idr = rcp_approx(dr);
        float yr[N];
#pragma unroll
        for (int j = 0; j < N; ++j) yr[j] = hr[j] * idr;
        const float ys = hs * idr;
        st_row(Y + r * N, yr);
        yv[r] = ys;
        st_row(a.K + gs * N * N + r * N, yr, -1.f);
        a.k[gs * N + r] = -ys;
    }
    g.sync();
    // (e) P -= H^T Y, p -= H^T y (column r of H against the rows of Y);
    // Abar = A - B Y, bbar = c - B y (row r of B against the rows of Y)
    float* Pt = scr + S::Pt;
    if (row) {
        float ab[N];
        ld_row(ab, st + L::A + r * N);
        float bb = st[L::c + r];
#pragma unroll 1
        for (int q = 0; q < N / 4; ++q) {
            const float4 b4 = reinterpret_cast<const float4*>(st + L::B + r * N)[q];
            const float4 y4 = reinterpret_cast<const float4*>(yv)[q];
            const float bq[4] = {b4.x, b4.y, b4.z, b4.w}, yq[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int l = 4 * q + i;
                const float hlr = H[l * N + r];
                float yl[N];
                ld_row(yl, Y + l * N);
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    pn[j] = fmaf(-hlr, yl[j], pn[j]);
                    ab[j] = fmaf(-bq[i], yl[j], ab[j]);
                }
                ps = fmaf(-hlr, yq[i], ps);
                bb = fmaf(-bq[i], yq[i], bb);
            }
        }
        st_row(Pt + r * N, pn);
        st_row(a.Abar + gs * N * N + r * N, ab);
        a.bbar[gs * N + r] = bb;
        if (abar_sm) {             // also left in shared memory: rows, then bbar
            st_row(abar_sm + r * N, ab);
            abar_sm[N * N + r] = bb;
        }
    }
    g.sync();
    // (f) P <- (P + P^T) / 2, the value function of the next step
    if (row) {
        float Pn[N];
#pragma unroll
        for (int j = 0; j < N; ++j) Pn[j] = 0.5f * (pn[j] + Pt[j * N + r]);
        st_row(scr + S::V + r * N, Pn);
        scr[S::vp + r] = ps;
        st_row(a.P + gs * N * N + r * N, Pn);
        a.p[gs * N + r] = ps;
    }
    return ok;
}

// ----------------------------------------- linearisation, one robot, rows
// Entry c of {v0, v1, v2} for a lane-dependent c, by selects (a dynamic
// index into a register array would go through local memory).
__device__ __forceinline__ float pick3(float v0, float v1, float v2, int c)
{
    return c == 0 ? v0 : (c == 1 ? v1 : v2);
}

// Row a of the cross-product matrix [v]x (rows (0, -v2, v1), (v2, 0, -v0),
// (-v1, v0, 0)), a lane-dependent.
__device__ __forceinline__ void skew_row(const float (&v)[3], int a, float (&o)[3])
{
    o[0] = a == 1 ? v[2] : (a == 2 ? -v[1] : 0.f);
    o[1] = a == 0 ? -v[2] : (a == 2 ? v[0] : 0.f);
    o[2] = a == 0 ? v[1] : (a == 1 ? -v[0] : 0.f);
}

// One stage of the single-robot SRBD linearisation (Sec. II-B, II-F) by the
// 16 lanes of a half-warp: lane r < 12 writes row r of A, B, Q and R and
// c_r, q_r, r_r into st (StageL<12, 12>) from the closed-form derivatives of
// srbd_linearize_stage, selecting its row's terms instead of branching on r,
// so that the lanes stay converged:
//   A = I + dt df/dx:  rows 0..5: e_r + dt e_{r+6} (p' = v, theta' = w);
//     rows 9..11 (a = r - 9): e_r + dt I_a^-1 ([F]x row a at p, -([w]x I -
//     [I w]x) row a at w), F = sum of the stance forces;
//   B = dt df/du:  rows 6..8: dt / mass at the stance feet's component r - 6;
//     rows 9..11: dt I_a^-1 [foot_j - p]x row a at stance foot j;
//   c_r = (x_r - x_{k+1, r}) + dt f_r(x, u);
//   Q = diag(W) (W_N at the terminal), q_r = W_r (x_r - xref_r) - lam_{k,r};
//   R = diag(W_u) + the barrier curvature of the friction pyramid (3 x 3
//   block of the lane's foot), r_r = W_u,r (u_r - uref_r) + barrier slope.
// The costate terms A^T lam_{k+1} of q and B^T lam_{k+1} of r are left out:
// riccati_rows adds lam_{k+1} to p' + P'c, which both terms multiply.  The
// model inputs come from an input buffer filled by SrbdSource::fetch (x, x1,
// lam_k, lam_{k+1}, xref, u, uref, contact); nothing is read at the terminal
// beyond x, lam_k and xref.
__device__ __forceinline__ void srbd_lin_rows12(const Grp<16>& g, float* st,
                                                const pdilqr_srbd_model& md, const float* in,
                                                bool terminal)
{
    using L = StageL<12, 12>;
    const int r = g.t;
    if (r >= 12) return;
    const float* x = in;
    const float* x1 = in + 12;
    const float* l0 = in + 24;
    const float* xr = in + 48;
    const float* u = in + 60;
    const float* ur = in + 72;
    const uint8_t* ct = reinterpret_cast<const uint8_t*>(in + 84);
    float row[12];
    // the lane's weights, read with static indices (a lane-dependent index
    // into the kernel parameters would serialise the lanes' constant-cache
    // reads) and selected
    float wq = 0.f, wu = 0.f;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
        wq = j == r ? (terminal ? md.WN[j] : md.W[j]) : wq;
        wu = j == r ? md.Wu[j] : wu;
    }
    // Q row r and q_r
#pragma unroll
    for (int j = 0; j < 12; ++j) row[j] = j == r ? wq : 0.f;
    st_row(st + L::Q + r * 12, row);
    st[L::q + r] = wq * (x[r] - xr[r]) - l0[r];
    if (terminal) return;

    const float dt = md.dt;
    float p[3], w[3], sv[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) { p[i] = x[i]; w[i] = x[9 + i]; }
#pragma unroll
    for (int j = 0; j < 4; ++j) sv[j] = ct[j] ? 1.f : 0.f;
    // stance force sum F and torque sum tau = sum_j s_j (foot_j - p) x f_j
    float F[3] = {0.f, 0.f, 0.f}, tau[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float f[3] = {u[3 * j] * sv[j], u[3 * j + 1] * sv[j], u[3 * j + 2] * sv[j]};
        const float arm[3] = {md.foot[j][0] - p[0], md.foot[j][1] - p[1], md.foot[j][2] - p[2]};
        float t[3];
        cross3f(arm, f, t);
#pragma unroll
        for (int i = 0; i < 3; ++i) { F[i] += f[i]; tau[i] += t[i]; }
    }
    const float Iw[3] = {md.inertia[0] * w[0], md.inertia[1] * w[1], md.inertia[2] * w[2]};
    float gyro[3];
    cross3f(w, Iw, gyro);
    const bool ang = r >= 9, lin = r >= 6 && r < 9;
    const int a = ang ? r - 9 : 0;      // angular row's axis
    const int b = lin ? r - 6 : 0;      // linear-velocity row's axis
    const float Ia = pick3(md.inertia[0], md.inertia[1], md.inertia[2], a);
    const float sc = dt * rcp_approx(Ia);
    const float dtm = dt * rcp_approx(md.mass);
    // c_r = (x_r - x1_r) + dt f_r
    float fr;
    if (r < 6) fr = x[r + 6];
    else if (lin) fr = pick3(F[0], F[1], F[2], b) / md.mass - (b == 2 ? md.gravity : 0.f);
    else fr = (pick3(tau[0], tau[1], tau[2], a) - pick3(gyro[0], gyro[1], gyro[2], a)) / Ia;
    st[L::c + r] = (x[r] - x1[r]) + dt * fr;
    // A row r
    {
        float sF[3], sw[3], sIw[3];
        skew_row(F, a, sF);
        skew_row(w, a, sw);
        skew_row(Iw, a, sIw);
#pragma unroll
        for (int j = 0; j < 12; ++j) row[j] = (j == r ? 1.f : 0.f) + (r < 6 && j == r + 6 ? dt : 0.f);
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            row[l] += ang ? sc * sF[l] : 0.f;
            row[9 + l] -= ang ? sc * (sw[l] * md.inertia[l] - sIw[l]) : 0.f;
        }
        st_row(st + L::A + r * 12, row);
    }
    // B row r
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float arm[3] = {md.foot[j][0] - p[0], md.foot[j][1] - p[1], md.foot[j][2] - p[2]};
        float sa[3];
        skew_row(arm, a, sa);
#pragma unroll
        for (int l = 0; l < 3; ++l)
            row[3 * j + l] = sv[j] * (ang ? sc * sa[l] : (lin && l == b ? dtm : 0.f));
    }
    st_row(st + L::B + r * 12, row);
    // R row r and r_r: control r is component cp of foot jf
    const int jf = r / 3, cp = r - 3 * jf;
#pragma unroll
    for (int j = 0; j < 12; ++j) row[j] = j == r ? wu : 0.f;
    float grad = wu * (u[r] - ur[r]);
    if (ct[jf]) {
        const float f0 = u[3 * jf], f1 = u[3 * jf + 1], f2 = u[3 * jf + 2];
        const float mu = md.mu_fric;
        float blk[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const float g0 = cone_g(c, 0, mu), g1 = cone_g(c, 1, mu), g2 = cone_g(c, 2, mu);
            const float xi = g0 * f0 + g1 * f1 + g2 * f2;
            const bool hi = xi >= md.bar_delta;
            const float iv = rcp_approx(hi ? xi : md.bar_delta);
            const float d1 = hi ? -md.bar_mu * iv : md.bar_mu * (xi - 2.f * md.bar_delta) * iv * iv;
            const float d2 = md.bar_mu * iv * iv;
            const float gc = pick3(g0, g1, g2, cp);
            grad += d1 * gc;
            blk[0] += d2 * gc * g0;
            blk[1] += d2 * gc * g1;
            blk[2] += d2 * gc * g2;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int l = 0; l < 3; ++l) row[3 * j + l] += j == jf ? blk[l] : 0.f;
    }
    st_row(st + L::R + r * 12, row);
    st[L::r + r] = grad;
}

// ------------------------------------------------------ merit, one half
// SRBD dynamics along a search direction: f(x + a dx, u + a du) of one robot
// is exactly quadratic in a (the torques (foot - p) x f are bilinear in
// position and force, the gyroscopic term w x I w is quadratic in w), so
// f(a) = f0 + a f1 + a^2 f2 with
//   f0 = f(x, u),
//   f1 = (dv, dw, sum s_j df_j / m,
//         I^-1 (sum s_j ((foot_j - p) x df_j - dp x f_j) - dw x I w - w x I dw)),
//   f2 = (0, 0, 0, I^-1 (- sum s_j dp x df_j - dw x I dw)).
__device__ __forceinline__ void srbd_xdot_poly(const pdilqr_srbd_model& md, const float* x,
                                               const float* u, const float* dx, const float* du,
                                               const uint8_t* s, float* f0, float* f1, float* f2)
{
    srbd_xdot(md, x, u, s, f0);
    const float* p = x;
    const float* w = x + 9;
    const float* dp = dx;
    const float* dw = dx + 9;
    float fs[3] = {0.f, 0.f, 0.f}, t1[3] = {0.f, 0.f, 0.f}, t2[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (!s[j]) continue;
        const float* f = u + 3 * j;
        const float* df = du + 3 * j;
        const float arm[3] = {md.foot[j][0] - p[0], md.foot[j][1] - p[1], md.foot[j][2] - p[2]};
        float a1[3], a2[3], a3[3];
        cross3f(arm, df, a1);
        cross3f(dp, f, a2);
        cross3f(dp, df, a3);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            fs[i] += df[i];
            t1[i] += a1[i] - a2[i];
            t2[i] -= a3[i];
        }
    }
    const float Iw[3] = {md.inertia[0] * w[0], md.inertia[1] * w[1], md.inertia[2] * w[2]};
    const float Idw[3] = {md.inertia[0] * dw[0], md.inertia[1] * dw[1], md.inertia[2] * dw[2]};
    float g1[3], g2[3], g3[3];
    cross3f(dw, Iw, g1);
    cross3f(w, Idw, g2);
    cross3f(dw, Idw, g3);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        f1[i] = dx[6 + i];
        f1[3 + i] = dw[i];
        f1[6 + i] = fs[i] / md.mass;
        f1[9 + i] = (t1[i] - g1[i] - g2[i]) / md.inertia[i];
        f2[i] = 0.f;
        f2[3 + i] = 0.f;
        f2[6 + i] = 0.f;
        f2[9 + i] = (t2[i] - g3[i]) / md.inertia[i];
    }
}

// Compensated FP32 accumulation (Knuth's TwoSum): hi + lo carries the sum to
// about twice FP32 precision, which keeps per-lane sums of stage terms as
// accurate as FP64 accumulation without the FP64 pipe.
__device__ __forceinline__ void acc2(float& hi, float& lo, float v)
{
    const float s = hi + v;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (v - bp);
    hi = s;
}

// The line-search merit of merit_block ([0] J(0), [1] theta(0), [2] dphi,
// [3 + t] J(a_t) - J(0), [13 + t] theta(a_t), [23] |dz|_inf, [25] |x|_inf)
// for one single-robot instance (n = m = 12) by a 16-lane half (stages
// kfirst + lane, + kstep, ...: several halves may split an instance, each
// writing its own sums to its `out`), for the step sizes a_t = 2^-t with
// T0 <= t <= T1 (and, when T0 = 0, the current
// point and the norms); slots of other step sizes are left untouched.
// Every lane takes whole stages (k = lane, lane + 16, ...) and reads each
// stage's data once: the tracking terms of J(a) - J(0) are the polynomial
// a A1 + a^2 A2 with A1 = sum W dx (x - xref) + sum Wu du (u - uref) and
// A2 = sum (W dx^2 + Wu du^2) / 2 (the sum the stage-wise form
// a dx (e + a dx / 2) adds up), the defect x_{k+1} - h(x_k + a dx_k, u_k +
// a du_k) is (x_{k+1} - x_k - dt f0) + a (dx_{k+1} - dx_k - dt f1) - a^2 dt
// f2 (srbd_xdot_poly), and the friction-pyramid barriers are differenced per
// step size without cancellation (barrier_diff), the step sizes of a row
// independent of one another.  Each lane sums its stages in compensated FP32
// (hi, lo pairs in shared memory, acc: 16 x 46 floats); the lanes' sums are
// added in FP64 at the end.
template <int T0, int T1>
__device__ void merit_rows(const Grp<16>& g, const pdilqr_srbd_model& md, const float* x,
                           const float* u, const float* dx, const float* du, const float* xr,
                           const float* ur, const uint8_t* ct, const float* x0hat, int N,
                           float* acc, float* fbuf, double* out, int kfirst = 0, int kstep = 16)
{
    constexpr int NS = 23;            // summed slots: out[0..22]
    constexpr int NT = T1 - T0 + 1;   // step sizes evaluated
    constexpr bool CUR = T0 == 0;     // also the current point
    float* my = acc + g.t * 2 * NS;   // (hi, lo) of slot s at my[2 s], my[2 s + 1]
    for (int i = 0; i < 2 * NS; ++i) my[i] = 0.f;
    auto add = [&](int slot, float v) { acc2(my[2 * slot], my[2 * slot + 1], v); };
    float step = 0.f, xmax = 0.f;
    for (int k = kfirst + g.t; k <= N; k += kstep) {
        const bool term = k == N;
        const float* Wx = term ? md.WN : md.W;
        float A1 = 0.f, A2 = 0.f, J0 = 0.f, th0 = 0.f;
        float th[NT];                     // theta terms of the step sizes
        float e0[12], e1[12], e2[12];     // defect polynomial (not used at the terminal stage)
        float uk[12], duk[12];
#pragma unroll
        for (int t = 0; t < NT; ++t) th[t] = 0.f;
        {
            float xk[12], dxk[12];
            ld_row(xk, x + (int64_t)k * 12);
            ld_row(dxk, dx + (int64_t)k * 12);
            {
                float xrk[12];
                ld_row(xrk, xr + (int64_t)k * 12);
#pragma unroll
                for (int i = 0; i < 12; ++i) {
                    const float e = xk[i] - xrk[i];
                    A1 = fmaf(Wx[i] * dxk[i], e, A1);
                    A2 = fmaf(0.5f * Wx[i] * dxk[i], dxk[i], A2);
                    J0 = fmaf(0.5f * Wx[i] * e, e, J0);
                    step = fmaxf(step, fabsf(dxk[i]));
                    xmax = fmaxf(xmax, fabsf(xk[i]));
                }
            }
            if (k == 0) {
                // initial-state term |xhat_0 - (x_0 + a dx_0)| of theta
                float h0[12];
                ld_row(h0, x0hat);
                float ss0 = 0.f;
#pragma unroll
                for (int i = 0; i < 12; ++i) ss0 = fmaf(h0[i] - xk[i], h0[i] - xk[i], ss0);
                th0 = sqrtf(ss0);
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const float a = 1.f / (float)(1 << (T0 + t));
                    float ss = 0.f;
#pragma unroll
                    for (int i = 0; i < 12; ++i) {
                        const float d = h0[i] - fmaf(a, dxk[i], xk[i]);
                        ss = fmaf(d, d, ss);
                    }
                    th[t] = sqrtf(ss);
                }
            }
            if (!term) {
                ld_row(uk, u + (int64_t)k * 12);
                ld_row(duk, du + (int64_t)k * 12);
                float x1[12], dx1[12];
                {
                    float urk[12];
                    ld_row(urk, ur + (int64_t)k * 12);
#pragma unroll
                    for (int i = 0; i < 12; ++i) {
                        const float eu = uk[i] - urk[i];
                        A1 = fmaf(md.Wu[i] * duk[i], eu, A1);
                        A2 = fmaf(0.5f * md.Wu[i] * duk[i], duk[i], A2);
                        J0 = fmaf(0.5f * md.Wu[i] * eu, eu, J0);
                        step = fmaxf(step, fabsf(duk[i]));
                    }
                }
                srbd_xdot_poly(md, xk, uk, dxk, duk, ct + (int64_t)k * 4, e0, e1, e2);
                ld_row(x1, x + (int64_t)(k + 1) * 12);
                ld_row(dx1, dx + (int64_t)(k + 1) * 12);
#pragma unroll
                for (int i = 0; i < 12; ++i) {
                    e0[i] = (x1[i] - xk[i]) - md.dt * e0[i];
                    e1[i] = (dx1[i] - dxk[i]) - md.dt * e1[i];
                    e2[i] = -md.dt * e2[i];
                }
            }
        }
        float cj[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const float a = 1.f / (float)(1 << (T0 + t));
            cj[t] = a * A1 + a * a * A2;
        }
        float dphi = A1;
        if (!term) {
            const uint8_t* ck = ct + (int64_t)k * 4;
            float* fu = fbuf + 24 * g.t;   // forces and steps, read back by foot index
            st_row(fu, uk);
            st_row(fu + 12, duk);
            // friction-pyramid barriers of the stance feet
#pragma unroll 1
            for (int j = 0; j < 4; ++j) {
                if (!ck[j]) continue;
                const float f0 = fu[3 * j], f1 = fu[3 * j + 1], f2 = fu[3 * j + 2];
                const float d0 = fu[12 + 3 * j], d1 = fu[13 + 3 * j], d2 = fu[14 + 3 * j];
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    const float g0 = cone_g(c, 0, md.mu_fric), g1 = cone_g(c, 1, md.mu_fric),
                                g2 = cone_g(c, 2, md.mu_fric);
                    const float xi = g0 * f0 + g1 * f1 + g2 * f2;
                    const float dxi = g0 * d0 + g1 * d1 + g2 * d2;
                    if (CUR) {
                        float v, s1;
                        barrier_vs(xi, md.bar_mu, md.bar_delta, v, s1);
                        J0 += v;
                        dphi = fmaf(s1, dxi, dphi);
                    }
#pragma unroll
                    for (int t = 0; t < NT; ++t)
                        cj[t] += barrier_diff(xi, dxi / (float)(1 << (T0 + t)), md.bar_mu, md.bar_delta);
                }
            }
            // defects |x_{k+1} - h(x_k + a dx_k, u_k + a du_k)|
            if (CUR) {
                float ss = 0.f;
#pragma unroll
                for (int i = 0; i < 12; ++i) ss = fmaf(e0[i], e0[i], ss);
                th0 += sqrtf(ss);
            }
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const float a = 1.f / (float)(1 << (T0 + t));
                float ss = 0.f;
#pragma unroll
                for (int i = 0; i < 12; ++i) {
                    const float ei = fmaf(a, fmaf(a, e2[i], e1[i]), e0[i]);
                    ss = fmaf(ei, ei, ss);
                }
                th[t] += sqrtf(ss);
            }
        }
        if (CUR) {
            add(0, J0);
            add(1, th0);
            add(2, dphi);
        }
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            add(3 + T0 + t, cj[t]);
            add(13 + T0 + t, th[t]);
        }
    }
    if (CUR) {
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            step = fmaxf(step, __shfl_xor_sync(g.mask, step, o, 16));
            xmax = fmaxf(xmax, __shfl_xor_sync(g.mask, xmax, o, 16));
        }
    }
    g.sync();
    for (int s = g.t; s < NS; s += 16) {
        const bool mine = (s >= 3 + T0 && s <= 3 + T1) || (s >= 13 + T0 && s <= 13 + T1) || (CUR && s < 3);
        if (!mine) continue;
        double v = 0.0;
        for (int l = 0; l < 16; ++l) v += (double)acc[l * 2 * NS + 2 * s] + (double)acc[l * 2 * NS + 2 * s + 1];
        out[s] = v;
    }
    if (CUR && g.t == 0) {
        out[23] = (double)step;
        out[25] = (double)xmax;
    }
    g.sync();
}

// The step sizes 2^-1 .. 2^-9, needed only when the full step is rejected:
// kept out of line so that the common path keeps its registers.
static __device__ __noinline__ void merit_rows_rest(const Grp<16>& g, const pdilqr_srbd_model& md,
                                                    const float* x, const float* u, const float* dx,
                                                    const float* du, const float* xr, const float* ur,
                                                    const uint8_t* ct, const float* x0hat, int N,
                                                    float* acc, float* fbuf, double* out,
                                                    int kfirst = 0, int kstep = 16)
{
    merit_rows<1, 9>(g, md, x, u, dx, du, xr, ur, ct, x0hat, N, acc, fbuf, out, kfirst, kstep);
}

// Forward rollout of stages [k0, k1) of an instance at slot offset off with
// horizon N, rows per lane: dx_{k+1} = Abar dx_k + bbar, du_k = K dx_k + k_k,
// dlam_k = P dx_k + p_k (du_N = 0), from dx_{k0} (lane r < n holds its entry
// r in xv0); the rows of K, P, Abar were written by the same lanes in the
// backward sweep, and the rows of stage k + 1 are loaded while stage k is
// applied.  xs: 16 floats of shared memory (the state broadcast).  Returns
// false on a lane that wrote a non-finite value.
template <int NX>
__device__ bool rollout_rows(const Grp<16>& g, const KktArgs& ka, int64_t off, int N, int k0,
                             int k1, float xv0, float* xs)
{
    constexpr int NU = NX;
    const int r = g.t;
    const bool row = r < NX;
    float* dx = ka.dx + off * NX;
    float* du = ka.du + off * NU;
    float* dl = ka.dlam + off * NX;
    float xv = xv0;
    bool fin = true;
    float Kc[NX], Pc[NX], Ac[NX], kc = 0.f, pc = 0.f, bc = 0.f;
#pragma unroll
    for (int j = 0; j < NX; ++j) { Kc[j] = 0.f; Pc[j] = 0.f; Ac[j] = 0.f; }
    if (row && k0 < k1) {
        const int64_t gs = off + k0;
        ld_row(Pc, ka.P + gs * NX * NX + r * NX);
        pc = ka.p[gs * NX + r];
        if (k0 < N) {
            ld_row(Kc, ka.K + gs * NU * NX + r * NX);
            ld_row(Ac, ka.Abar + gs * NX * NX + r * NX);
            kc = ka.k[gs * NU + r];
            bc = ka.bbar[gs * NX + r];
        }
    }
    for (int k = k0; k < k1; ++k) {
        const int64_t gs = off + k;
        float Kn[NX], Pn[NX], An[NX], kn = 0.f, pn = 0.f, bn = 0.f;
#pragma unroll
        for (int j = 0; j < NX; ++j) { Kn[j] = 0.f; Pn[j] = 0.f; An[j] = 0.f; }
        if (row && k + 1 < k1) {
            ld_row(Pn, ka.P + (gs + 1) * NX * NX + r * NX);
            pn = ka.p[(gs + 1) * NX + r];
            if (k + 1 < N) {
                ld_row(Kn, ka.K + (gs + 1) * NU * NX + r * NX);
                ld_row(An, ka.Abar + (gs + 1) * NX * NX + r * NX);
                kn = ka.k[(gs + 1) * NU + r];
                bn = ka.bbar[(gs + 1) * NX + r];
            }
        }
        if (row) xs[r] = xv;
        g.sync();
        if (row) {
            float xl[NX];
            ld_row(xl, xs);
            float lv = pc, uv = kc, nv = bc;
#pragma unroll
            for (int j = 0; j < NX; ++j) {
                lv = fmaf(Pc[j], xl[j], lv);
                uv = fmaf(Kc[j], xl[j], uv);
                nv = fmaf(Ac[j], xl[j], nv);
            }
            dx[(int64_t)k * NX + r] = xv;
            dl[(int64_t)k * NX + r] = lv;
            du[(int64_t)k * NU + r] = k < N ? uv : 0.f;
            fin = fin && isfinite(xv) && isfinite(lv) && (k == N || isfinite(uv));
            xv = nv;
        }
        g.sync();   // xs is rewritten at the next stage
#pragma unroll
        for (int j = 0; j < NX; ++j) { Pc[j] = Pn[j]; Kc[j] = Kn[j]; Ac[j] = An[j]; }
        pc = pn; kc = kn; bc = bn;
    }
    return fin;
}

// Linearise the stage whose inputs are in `in` into st: the one-robot row
// form (costate terms left to the Riccati step) at n = 12, else the generic
// row-parallel linearisation.  PENDING: copy groups committed after this
// stage's.
template <int NX, int PENDING>
__device__ __forceinline__ void lin_stage(const Grp<16>& g, const SrbdSource& src, float* st,
                                          const float* in, bool terminal)
{
    if constexpr (NX == 12) {
        cp_async_wait<PENDING>();
        g.sync();
        srbd_lin_rows12(g, st, src.md, in, terminal);
        g.sync();
    } else {
        src.template linearize<NX, NX, 16, PENDING>(g, st, in, terminal);
    }
}

// ------------------------------------------------------------- the kernel
template <int NX>
struct SqpRowsSmem {
    using L = StageL<NX, NX>;
    static constexpr int ST = 0;                              // stage (StageL layout)
    static constexpr int SCR = round4(ST + L::SIZE);          // Riccati scratch
    static constexpr int INB = SCR + RowRicL<NX>::SIZE;       // two stage-input buffers
    static constexpr int INF = round4(SrbdSource::in_floats<NX, NX>());
    static constexpr int XS = INB + 2 * INF;                  // rollout state, 16 floats
    static constexpr int MER = XS + 16;                       // merit: 26 doubles
    static constexpr int CTL = MER + 2 * 26;                  // step size, stop and full-step flags
    static constexpr int PER = round4(CTL + 4);               // one half (instance)
    static constexpr size_t BYTES = 2 * PER * sizeof(float);
    // the merit's per-lane sums (16 x 46 floats) reuse the stage area and
    // its per-lane force buffers (16 x 24 floats) the Riccati scratch
    static_assert(L::SIZE >= 16 * 46, "merit sums fit the stage area");
    static_assert(RowRicL<NX>::SIZE >= 16 * 24, "merit force buffers fit the scratch");
};

// The fused SQP with the sequential recursion for the SRBD model with n =
// m = NX: CTAs of one warp, two instances (consecutive entries of the
// longest-first order, so mostly equal horizons) per warp.  Per iteration
// and instance: the backward sweep (linearisation of stage k, then the
// row-per-lane Riccati step), the forward rollout dx_{k+1} = Abar dx_k +
// bbar, du = K dx + k, dlam = P dx + p, the merit of the ten step sizes, the
// filter decision of Sec. II-E and the update of Eq. (linear_rollout).
template <int NX>
__device__ __forceinline__ void sqp_rows_instance(const SqpArgs& a, const Grp<16>& g, float* base,
                                                  int inst)
{
    using SM = SqpRowsSmem<NX>;
    using L = StageL<NX, NX>;
    constexpr int NU = NX;
    const int r = g.t;
    const bool row = r < NX;
    float* st = base + SM::ST;
    float* scr = base + SM::SCR;
    float* xs = base + SM::XS;
    double* mer = reinterpret_cast<double*>(base + SM::MER);
    float* alpha_sh = base + SM::CTL;
    int* ctl = reinterpret_cast<int*>(base + SM::CTL + 1);

    const KktArgs& ka = a.ka;
    const int N = ka.N[inst];
    const int64_t off = ka.off[inst];
    const int nrob = a.md.nrob;
    const SrbdSource src{a.md, a.x, a.u, a.lam, a.xref, a.uref, a.contact, nrob, nullptr};
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

    int status = ST_OK, iters = 0;
    for (int it = 0; it < a.max_iters; ++it) {
        // ---- backward sweep: terminal value function, then Eq. (lqr) from k = N - 1 down
        // stage inputs are fetched one stage ahead into alternating buffers
        float* inb = base + SM::INB;
        src.template fetch<NX, NU, 16>(g, inb + (N & 1) * SM::INF, off + N, true);
        if (N >= 1) src.template fetch<NX, NU, 16>(g, inb + ((N - 1) & 1) * SM::INF, off + N - 1, false);
        lin_stage<NX, 1>(g, src, st, inb + (N & 1) * SM::INF, true);
        if (row) {
            float PN[NX];
            ld_row(PN, st + L::Q + r * NX);
            const float pN = st[L::q + r];
            st_row(scr + RowRicL<NX>::V + r * NX, PN);
            scr[RowRicL<NX>::vp + r] = pN;
            st_row(ka.P + (off + N) * NX * NX + r * NX, PN);
            ka.p[(off + N) * NX + r] = pN;
        }
        bool ok = true;
        for (int k = N - 1; k >= 0; --k) {
            g.sync();   // every read of the previous stage is done
            const float* ink = inb + (k & 1) * SM::INF;
            if (k >= 1) {
                src.template fetch<NX, NU, 16>(g, inb + ((k - 1) & 1) * SM::INF, off + k - 1, false);
                lin_stage<NX, 1>(g, src, st, ink, false);
            } else {
                lin_stage<NX, 0>(g, src, st, ink, false);
            }
            // lam_{k+1} of the input buffer when the linearisation left out
            // the costate terms (the one-robot row form)
            const float* l1 = NX == 12 ? ink + 3 * 12 : nullptr;
            ok = riccati_rows<NX>(g, st, scr, ka, off + k, false, nullptr, l1) && ok;
        }
        if (!ok) {
            status = ST_NOT_SPD;
            break;
        }
        // ---- forward rollout from dx_0 = xhat_0 - x_0
        const bool fin = rollout_rows<NX>(g, ka, off, N, 0, N + 1, row ? xh[r] - x[r] : 0.f, xs);
        if (__any_sync(g.mask, !fin)) {
            status = ST_NONFINITE;
            break;
        }
        __threadfence_block();
        g.sync();
        iters = it + 1;
        // ---- line search (Sec. II-E): merit of the ten step sizes, filter
        // The full step first: the filter takes the largest accepted step
        // size, so the other nine are evaluated only when a = 1 is rejected
        // (or a replayed step asks for one of them); the step taken is the
        // one an evaluation of all ten would pick.
        merit_rows<0, 0>(g, a.md, x, u, dx, du, xr, ur, ct, xh, N, st, scr, mer);
        if (g.t == 0) {
            if (it == 0) mer[24] = (double)a.theta_frac * fmax(1.0, mer[1]);
            const bool full = a.alpha_replay ? a.alpha_replay[(int64_t)inst * a.max_iters + it] == 1.f
                                             : filter_ok(mer[1], mer[2], mer[24], 1.0, mer[3], mer[13], a.c_armijo);
            ctl[1] = full ? 1 : 0;
        }
        g.sync();
        if (!ctl[1]) merit_rows_rest(g, a.md, x, u, dx, du, xr, ur, ct, xh, N, st, scr, mer);
        if (g.t == 0) {
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
            // no step accepted while theta(0) sits at the rounding floor of
            // the FP32 iterate: converged at working precision
            const double floor_th = (double)(N + 1) * sqrt((double)NX) * 0x1p-23 * fmax(1.0, mer[25]);
            const bool at_floor = alpha == 0.f && th0 <= floor_th && !a.alpha_replay;
            alpha_sh[0] = at_floor ? -1.f : alpha;
            ctl[0] = (at_floor || (mer[23] < (double)a.tol_step && th_new < (double)a.tol_theta)) ? 1 : 0;
            if (a.alpha) a.alpha[(int64_t)inst * a.max_iters + it] = alpha;
        }
        g.sync();
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
            for (int e = g.t; e < (N + 1) * NX / 4; e += 16) {
                float4 v = x4[e], d = dx4[e];
                v.x += alpha * d.x; v.y += alpha * d.y; v.z += alpha * d.z; v.w += alpha * d.w;
                x4[e] = v;
                v = l4[e]; d = dl4[e];
                v.x += alpha * d.x; v.y += alpha * d.y; v.z += alpha * d.z; v.w += alpha * d.w;
                l4[e] = v;
            }
            float4* u4 = reinterpret_cast<float4*>(u);
            const float4* du4 = reinterpret_cast<const float4*>(du);
            for (int e = g.t; e < N * NU / 4; e += 16) {
                float4 v = u4[e], d = du4[e];
                v.x += alpha * d.x; v.y += alpha * d.y; v.z += alpha * d.z; v.w += alpha * d.w;
                u4[e] = v;
            }
        }
        __threadfence_block();
        g.sync();
        if (ctl[0]) break;
    }
    if (a.J || a.theta) {
        // merit at the returned iterate (only the current-point column is read)
        merit_rows<0, 0>(g, a.md, x, u, dx, du, xr, ur, ct, xh, N, st, scr, mer);
    }
    if (g.t == 0) {
        a.iters[inst] = iters;
        a.status[inst] = status;
        if (a.J) a.J[inst] = mer[0];
        if (a.theta) a.theta[inst] = mer[1];
        if (a.alpha)
            for (int it = iters; it < a.max_iters; ++it) a.alpha[(int64_t)inst * a.max_iters + it] = 0.f;
    }
}


// CTAs of WPC warps, two instances (consecutive entries of the
// longest-first order) per warp, 2 WPC instances per CTA; the warps of a CTA
// share nothing but the CTA (an instance's half-warp synchronises only
// itself), so WPC sets the granularity of the hardware's CTA scheduling,
// which the batch autotuner picks.  8 / WPC CTAs per SM at 255 registers per
// thread (12 one-warp CTAs per SM at 168 registers spilled and were 16 %
// slower on the 4096-instance batch).  (A persistent form, a grid of the
// resident CTAs pulling pairs from a counter, measured the same on that
// batch and 4 % slower on one instance, its loop doubling the register
// spills; the hardware's CTA scheduling over the longest-first order already
// balances the batch, whose 2048 one-warp CTAs fit in 1.7 waves.)
template <int NX, int WPC>
__global__ void __launch_bounds__(32 * WPC, 8 / WPC) sqp_rows_kernel(const __grid_constant__ SqpArgs a)
{
    using SM = SqpRowsSmem<NX>;
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, h = lane >> 4, wp = threadIdx.x >> 5;
    const int slot = 2 * (blockIdx.x * WPC + wp) + h;
    if (slot >= a.ka.count) return;   // past the batch's end: this half runs nothing
    Grp<16> g{lane & 15, 0};
    g.mask = 0xffffu << (16 * h);
    sqp_rows_instance<NX>(a, g, smem + (2 * wp + h) * SM::PER, a.ka.order ? a.ka.order[slot] : slot);
}

}  // namespace pdl
