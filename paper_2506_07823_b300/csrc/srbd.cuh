// srbd.cuh -- single-rigid-body quadruped model on the GPU: per-stage
// linearisation (Sec. II-B, II-F) and the line-search merit (Sec. II-E).
//
// Model (one robot, x = [p, theta, v, omega], u = [f_0..f_3]):
//   p' = v, theta' = omega, v' = sum_j s_j f_j / mass - g e_z,
//   omega' = I^-1 ( sum_j s_j (foot_j - p) x f_j - omega x (I omega) ),
// one explicit Euler step of length dt; robots of a centralised problem are
// stacked and coupled only through the ring formation cost.
//
// The linearisation is row-parallel: thread i of the group produces row i
// of A, B, Q (state rows) or row i of R (control rows) from closed-form
// derivatives, so no thread waits on another until the costate terms
// A^T lam_{k+1}, B^T lam_{k+1} are added.
#pragma once

#include "kkt_scan.cuh"
#include "pdilqr.h"

namespace pdl {

// ------------------------------------------------------------ scalar parts
__device__ __forceinline__ void cross3f(const float* a, const float* b, float* o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// entry (r, c) of the cross-product matrix [a]x  ([a]x b = a x b)
__device__ __forceinline__ float skew_rc(const float* a, int r, int c)
{
    if (r == c) return 0.f;
    const int k = 3 - r - c;                       // the remaining axis
    const float sign = ((r + 1) % 3 == c) ? -1.f : 1.f;
    return sign * a[k];
}

// relaxed barrier (value, slope, curvature)
__device__ __forceinline__ void barrier3(float xi, float mu, float delta, float& v, float& d1,
                                         float& d2)
{
    if (xi >= delta) {
        v = -mu * logf(xi);
        d1 = -mu / xi;
        d2 = mu / (xi * xi);
    } else {
        const float t = (xi - 2.f * delta) / delta;
        v = 0.5f * mu * (t * t - 1.f) - mu * logf(delta);
        d1 = mu * t / delta;
        d2 = mu / (delta * delta);
    }
}

// B(xi + dxa) - B(xi) without cancellation between the two values
__device__ __forceinline__ float barrier_delta(float xi, float dxa, float mu, float delta)
{
    const float xn = xi + dxa;
    if (xi >= delta && xn >= delta) return -mu * log1pf(dxa / xi);
    if (xi < delta && xn < delta) return mu / (2.f * delta * delta) * dxa * (2.f * xi + dxa - 4.f * delta);
    float v0, v1, d;
    barrier3(xi, mu, delta, v0, d, d);
    barrier3(xn, mu, delta, v1, d, d);
    return v1 - v0;
}

// The relaxed barrier split as B(z) = -mu ln max(z, delta) + q(z), where
// q(z) = mu / (2 delta^2) (z - delta)(z - 3 delta) below delta and 0 above
// (the same function as barrier3: at z < delta, -mu ln delta + q(z) is the
// quadratic branch).  Branch-free forms of the value and slope, and of the
// difference B(xi + dxa) - B(xi): the log part is -mu log1p((max(xn, delta)
// - max(xi, delta)) / max(xi, delta)), whose argument is dxa itself when both
// points lie above delta, and the quadratic parts are differenced as
// mu / (2 delta^2) dxa (2 xi + dxa - 4 delta) when both lie below.
__device__ __forceinline__ void barrier_vs(float xi, float mu, float delta, float& v, float& d1)
{
    const float m = fmaxf(xi, delta);
    const float c = mu / (2.f * delta * delta);
    const bool lo = xi < delta;
    v = -mu * logf(m) + (lo ? c * (xi - delta) * (xi - 3.f * delta) : 0.f);
    d1 = lo ? 2.f * c * (xi - 2.f * delta) : -mu / m;
}

__device__ __forceinline__ float barrier_diff(float xi, float dxa, float mu, float delta)
{
    const float xn = xi + dxa;
    const float mi = fmaxf(xi, delta), mn = fmaxf(xn, delta);
    const bool li = xi < delta, ln = xn < delta;
    const float c = mu / (2.f * delta * delta);
    const float dm = (!li && !ln) ? dxa : mn - mi;
    const float lpart = -mu * log1pf(__fdividef(dm, mi));
    const float qi = c * (xi - delta) * (xi - 3.f * delta), qn = c * (xn - delta) * (xn - 3.f * delta);
    const float qpart = (li && ln) ? c * dxa * (2.f * xi + dxa - 4.f * delta) : (ln ? qn : 0.f) - (li ? qi : 0.f);
    return lpart + qpart;
}

// friction-pyramid row c of a stance foot: xi = G_c . f
__device__ __forceinline__ float cone_g(int c, int comp, float mu)
{
    // rows: mu fz + fx, mu fz - fx, mu fz + fy, mu fz - fy, fz
    if (comp == 2) return c < 4 ? mu : 1.f;
    if (comp == 0) return c == 0 ? 1.f : (c == 1 ? -1.f : 0.f);
    return c == 2 ? 1.f : (c == 3 ? -1.f : 0.f);
}

// time derivative of one robot's state (12) at (x, u) with stance flags s
__device__ __forceinline__ void srbd_xdot(const pdilqr_srbd_model& md, const float* x,
                                          const float* u, const uint8_t* s, float* xd)
{
    const float* p = x;
    const float* w = x + 9;
    float fs[3] = {0.f, 0.f, 0.f}, tau[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (!s[j]) continue;
        const float* f = u + 3 * j;
        const float arm[3] = {md.foot[j][0] - p[0], md.foot[j][1] - p[1], md.foot[j][2] - p[2]};
        float t[3];
        cross3f(arm, f, t);
#pragma unroll
        for (int i = 0; i < 3; ++i) { fs[i] += f[i]; tau[i] += t[i]; }
    }
    const float Iw[3] = {md.inertia[0] * w[0], md.inertia[1] * w[1], md.inertia[2] * w[2]};
    float gyro[3];
    cross3f(w, Iw, gyro);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        xd[i] = x[6 + i];
        xd[3 + i] = w[i];
        xd[6 + i] = fs[i] / md.mass - (i == 2 ? md.gravity : 0.f);
        xd[9 + i] = (tau[i] - gyro[i]) / md.inertia[i];
    }
}

// Component r of the time derivative of one robot's state.
__device__ __forceinline__ float srbd_xdot_comp(const pdilqr_srbd_model& md, const float* x,
                                                const float* u, const uint8_t* s, int r)
{
    if (r < 3) return x[6 + r];
    if (r < 6) return x[9 + (r - 3)];
    if (r < 9) {
        const int a = r - 6;
        float fs = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (s[j]) fs += u[3 * j + a];
        return fs / md.mass - (a == 2 ? md.gravity : 0.f);
    }
    const int a = r - 9, a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    const float* p = x;
    const float* w = x + 9;
    float tau = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (!s[j]) continue;
        const float* f = u + 3 * j;
        // ((foot_j - p) x f)_a
        tau += (md.foot[j][a1] - p[a1]) * f[a2] - (md.foot[j][a2] - p[a2]) * f[a1];
    }
    // (w x I w)_a
    const float gyro = w[a1] * md.inertia[a2] * w[a2] - w[a2] * md.inertia[a1] * w[a1];
    return (tau - gyro) / md.inertia[a];
}

// ------------------------------------------------------ stage linearisation
// Writes one stage in the StageL layout: A, B, c, Q, R, q, r (S = 0 is not
// written).  x1, l1 (next state / costate) are not read at the terminal.
template <int NX, int NU, int NT>
__device__ void srbd_linearize_stage(const Grp<NT>& g, float* st, const pdilqr_srbd_model& md,
                                     const float* x, const float* u, const float* x1,
                                     const float* l0, const float* l1, const float* xr,
                                     const float* ur, const uint8_t* ct, bool terminal)
{
    static_assert(NX % 12 == 0 && NU == NX, "SRBD stages hold whole robots");
    using L = StageL<NX, NU>;
    constexpr int NR = NX / 12;
    const float dt = md.dt;
    const float* Wx = terminal ? md.WN : md.W;
    const bool form = NR > 1;
    // state rows and control rows run on disjoint lanes of a warp
    constexpr int HALF = (NT == 32) ? 16 : NT;
    const int ts = (NT == 32) ? (g.t < 16 ? g.t : NX) : g.t;        // state-row lane
    const int tc = (NT == 32) ? (g.t >= 16 ? g.t - 16 : NU) : g.t;  // control-row lane
    // ---- state rows: A, B, c, Q, cost gradient in q
    for (int i = ts; i < NX; i += HALF) {
        const int b = i / 12, r = i % 12, o = 12 * b;
        const float* xb = x + o;
        float* Arow = st + L::A + i * NX;
        float* Brow = st + L::B + i * NU;
        float* Qrow = st + L::Q + i * NX;
        for (int j = 0; j < NX; ++j) Qrow[j] = 0.f;
        Qrow[i] = Wx[r];
        float grad = Wx[r] * (x[i] - xr[i]);
        if (form && r < 3) {
            const int an = (b + 1) % NR, ap = (b + NR - 1) % NR;
            const float e_self = xb[r] - x[12 * an + r] - md.d_form[b][r];
            const float e_prev = x[12 * ap + r] - xb[r] - md.d_form[ap][r];
            grad += md.w_form * (e_self - e_prev);
            Qrow[i] += 2.f * md.w_form;
            Qrow[12 * an + r] -= md.w_form;
            Qrow[12 * ap + r] -= md.w_form;
        }
        st[L::q + i] = grad;
        if (terminal) continue;
        const uint8_t* sb = ct + 4 * b;
        const float* ub = u + o;
        for (int j = 0; j < NX; ++j) Arow[j] = 0.f;
        for (int j = 0; j < NU; ++j) Brow[j] = 0.f;
        Arow[i] = 1.f;
        st[L::c + i] = (xb[r] - x1[i]) + dt * srbd_xdot_comp(md, xb, ub, sb, r);  // difference first
        if (r < 3) {
            Arow[o + 6 + r] = dt;
        } else if (r < 6) {
            Arow[o + 9 + (r - 3)] = dt;
        } else if (r < 9) {
            const int a = r - 6;
            const float dtm = dt * rcp_approx(md.mass);
            for (int j = 0; j < 4; ++j)
                if (sb[j]) Brow[o + 3 * j + a] = dtm;
        } else {
            const int a = r - 9;
            const float* p = xb;
            const float* w = xb + 9;
            const float sc = dt * rcp_approx(md.inertia[a]);
            const float Iw[3] = {md.inertia[0] * w[0], md.inertia[1] * w[1], md.inertia[2] * w[2]};
            for (int l = 0; l < 3; ++l) {
                // d omega'/d p = I^-1 sum_j s_j [f_j]x
                float fx = 0.f;
                for (int j = 0; j < 4; ++j)
                    if (sb[j]) fx += skew_rc(ub + 3 * j, a, l);
                Arow[o + l] += sc * fx;
                // d omega'/d omega = -I^-1 ([w]x I - [I w]x)
                Arow[o + 9 + l] -= sc * (skew_rc(w, a, l) * md.inertia[l] - skew_rc(Iw, a, l));
            }
            for (int j = 0; j < 4; ++j) {
                if (!sb[j]) continue;
                const float arm[3] = {md.foot[j][0] - p[0], md.foot[j][1] - p[1],
                                      md.foot[j][2] - p[2]};
                for (int l = 0; l < 3; ++l) Brow[o + 3 * j + l] = sc * skew_rc(arm, a, l);
            }
        }
    }
    // ---- control rows: R, cost gradient in r
    if (!terminal) {
        for (int i = tc; i < NU; i += HALF) {
            const int b = i / 12, r = i % 12, o = 12 * b, j = r / 3, comp = r % 3;
            float* Rrow = st + L::R + i * NU;
            for (int l = 0; l < NU; ++l) Rrow[l] = 0.f;
            Rrow[i] = md.Wu[r];
            float grad = md.Wu[r] * (u[i] - ur[i]);
            if (ct[4 * b + j]) {
                const float* f = u + o + 3 * j;
                for (int c = 0; c < 5; ++c) {
                    const float xi = cone_g(c, 0, md.mu_fric) * f[0] + cone_g(c, 1, md.mu_fric) * f[1] +
                                     cone_g(c, 2, md.mu_fric) * f[2];
                    // barrier slope and curvature (the value is not needed here)
                    float d1, d2;
                    if (xi >= md.bar_delta) {
                        const float ixi = rcp_approx(xi);
                        d1 = -md.bar_mu * ixi;
                        d2 = md.bar_mu * ixi * ixi;
                    } else {
                        const float idl = rcp_approx(md.bar_delta);
                        d1 = md.bar_mu * (xi - 2.f * md.bar_delta) * idl * idl;
                        d2 = md.bar_mu * idl * idl;
                    }
                    const float gc = cone_g(c, comp, md.mu_fric);
                    grad += d1 * gc;
                    for (int l = 0; l < 3; ++l)
                        Rrow[o + 3 * j + l] += d2 * gc * cone_g(c, l, md.mu_fric);
                }
            }
            st[L::r + i] = grad;
        }
    }
    g.sync();
    // ---- costate terms: q += A^T lam_{k+1} - lam_k, r += B^T lam_{k+1}
    if (!terminal) {
        mv<NX, NX, true, NT, false>(g, st + L::q, st + L::A, NX, l1, st + L::q);
        mv<NU, NX, true, NT, false>(g, st + L::r, st + L::B, NU, l1, st + L::r);
        g.sync();
    }
    for (int i = g.t; i < NX; i += NT) st[L::q + i] -= l0[i];
    g.sync();
}

// Source of LQ stages that linearises the SRBD model on the fly.
struct SrbdSource {
    const pdilqr_srbd_model& md;   // kernel parameter space (grid constant)
    const float *x, *u, *lam, *xref, *uref;
    const uint8_t* contact;
    int nrob;
    float* cache;                  // per-slot copy of linearised stages (or null)
    static constexpr bool kKeeps = true;

    // Keep a linearised stage (the LQ blocks, StageL::IN floats) so that the
    // Riccati sweep can stream it back instead of linearising again.
    template <int NX, int NU, int NT>
    __device__ __forceinline__ void keep(const Grp<NT>& g, const float* st, int64_t gs) const
    {
        constexpr int F = StageL<NX, NU>::IN;
        if (!cache) return;
        float4* dst = reinterpret_cast<float4*>(cache + gs * F);
        const float4* src = reinterpret_cast<const float4*>(st);
        for (int e = g.t; e < F / 4; e += NT) dst[e] = src[e];
    }
    template <int NX, int NU, int NT>
    __device__ __forceinline__ void reload(const Grp<NT>& g, float* st, int64_t gs) const
    {
        constexpr int F = StageL<NX, NU>::IN;
        if (!cache) {
            load<NX, NU, NT>(g, st, gs, false);
            return;
        }
        stage_copy<F, NT, true>(g.t, st, cache + gs * F);
        cp_async_commit();
        cp_async_wait_all();
        g.sync();
    }
    // Inputs of stage gs (x_k, x_{k+1}, lam_k, lam_{k+1}, xref_k, u_k, uref_k,
    // contact_k): fetch() issues their asynchronous copies into an input
    // buffer (IN_FLOATS floats, 16-byte aligned) and commits them as one
    // group; linearize() waits for the copies the thread issued, joins the
    // group and linearises the stage from the buffer into st.  load() is the
    // two back to back into the stage's own IN area.
    template <int NX, int NU>
    static constexpr int in_floats() { return 5 * round4(NX) + 2 * round4(NU) + round4(NX / 12 + 1); }
    template <int NX, int NU, int NT>
    __device__ __forceinline__ void fetch(const Grp<NT>& g, float* in, int64_t gs, bool terminal) const
    {
        constexpr int SX = round4(NX), SU = round4(NU);
        float* ix = in;
        float* ix1 = in + SX;
        float* il0 = in + 2 * SX;
        float* il1 = in + 3 * SX;
        float* ixr = in + 4 * SX;
        float* iu = in + 5 * SX;
        float* iur = iu + SU;
        uint8_t* ict = reinterpret_cast<uint8_t*>(iur + SU);
        stage_copy<NX, NT, true>(g.t, ix, x + gs * NX);
        stage_copy<NX, NT, true>(g.t, il0, lam + gs * NX);
        stage_copy<NX, NT, true>(g.t, ixr, xref + gs * NX);
        if (!terminal) {
            stage_copy<NX, NT, true>(g.t, ix1, x + (gs + 1) * NX);
            stage_copy<NX, NT, true>(g.t, il1, lam + (gs + 1) * NX);
            stage_copy<NU, NT, true>(g.t, iu, u + gs * NU);
            stage_copy<NU, NT, true>(g.t, iur, uref + gs * NU);
            // contact flags: nrob words of 4 bytes (4-byte aligned per stage)
            const float* csrc = reinterpret_cast<const float*>(contact + gs * 4 * nrob);
            for (int e = g.t; e < NX / 12; e += NT) {
                float* d = reinterpret_cast<float*>(ict) + e;
                if (__isShared(d)) cp_async4(d, csrc + e);
                else *d = csrc[e];      // stage area in the global workspace
            }
        }
        cp_async_commit();
    }
    // PENDING: copy groups this thread committed after the one to consume
    template <int NX, int NU, int NT, int PENDING = 0>
    __device__ __forceinline__ void linearize(const Grp<NT>& g, float* st, const float* in,
                                              bool terminal) const
    {
        constexpr int SX = round4(NX), SU = round4(NU);
        cp_async_wait<PENDING>();
        g.sync();
        const float* iu = in + 5 * SX;
        srbd_linearize_stage<NX, NU, NT>(g, st, md, in, iu, in + SX, in + 2 * SX, in + 3 * SX,
                                         in + 4 * SX, iu + SU,
                                         reinterpret_cast<const uint8_t*>(iu + 2 * SU), terminal);
    }
    template <int NX, int NU, int NT>
    __device__ __forceinline__ void load(const Grp<NT>& g, float* st, int64_t gs, bool terminal) const
    {
        float* in = st + StageL<NX, NU>::IN;
        fetch<NX, NU, NT>(g, in, gs, terminal);
        linearize<NX, NU, NT>(g, st, in, terminal);
    }
    __device__ __forceinline__ bool has_S() const { return false; }
};

// -------------------------------------------------------------- merit parts
// Stage cost l_k at (x, u) (terminal: u unused), FP32.
template <int NX>
__device__ float srbd_stage_cost(const pdilqr_srbd_model& md, const float* x, const float* u,
                                 const uint8_t* ct, const float* xr, const float* ur, bool terminal)
{
    constexpr int NR = NX / 12;
    const float* Wx = terminal ? md.WN : md.W;
    float J = 0.f;
    for (int i = 0; i < NX; ++i) {
        const float e = x[i] - xr[i];
        J += 0.5f * Wx[i % 12] * e * e;
    }
    if (NR > 1)
        for (int a = 0; a < NR; ++a)
            for (int r = 0; r < 3; ++r) {
                const float e = x[12 * a + r] - x[12 * ((a + 1) % NR) + r] - md.d_form[a][r];
                J += 0.5f * md.w_form * e * e;
            }
    if (terminal) return J;
    for (int i = 0; i < NX; ++i) {
        const float e = u[i] - ur[i];
        J += 0.5f * md.Wu[i % 12] * e * e;
    }
    for (int b = 0; b < NR; ++b)
        for (int j = 0; j < 4; ++j) {
            if (!ct[4 * b + j]) continue;
            const float* f = u + 12 * b + 3 * j;
            for (int c = 0; c < 5; ++c) {
                const float xi = cone_g(c, 0, md.mu_fric) * f[0] + cone_g(c, 1, md.mu_fric) * f[1] +
                                 cone_g(c, 2, md.mu_fric) * f[2];
                float v, d1, d2;
                barrier3(xi, md.bar_mu, md.bar_delta, v, d1, d2);
                J += v;
            }
        }
    return J;
}

// l_k(z + a dz) - l_k(z), evaluated term by term: quadratic terms as
// a d (e + a d / 2), barrier terms by barrier_delta.
template <int NX>
__device__ float srbd_stage_dcost(const pdilqr_srbd_model& md, const float* x, const float* u,
                                  const float* dx, const float* du, const uint8_t* ct,
                                  const float* xr, const float* ur, float a, bool terminal)
{
    constexpr int NR = NX / 12;
    const float* Wx = terminal ? md.WN : md.W;
    float d = 0.f;
    for (int i = 0; i < NX; ++i) d += Wx[i % 12] * a * dx[i] * ((x[i] - xr[i]) + 0.5f * a * dx[i]);
    if (NR > 1)
        for (int b = 0; b < NR; ++b)
            for (int r = 0; r < 3; ++r) {
                const int n2 = 12 * ((b + 1) % NR) + r;
                const float e = x[12 * b + r] - x[n2] - md.d_form[b][r];
                const float de = dx[12 * b + r] - dx[n2];
                d += md.w_form * a * de * (e + 0.5f * a * de);
            }
    if (terminal) return d;
    for (int i = 0; i < NX; ++i) d += md.Wu[i % 12] * a * du[i] * ((u[i] - ur[i]) + 0.5f * a * du[i]);
    for (int b = 0; b < NR; ++b)
        for (int j = 0; j < 4; ++j) {
            if (!ct[4 * b + j]) continue;
            const float* f = u + 12 * b + 3 * j;
            const float* df = du + 12 * b + 3 * j;
            for (int c = 0; c < 5; ++c) {
                const float g0 = cone_g(c, 0, md.mu_fric), g1 = cone_g(c, 1, md.mu_fric),
                            g2 = cone_g(c, 2, md.mu_fric);
                const float xi = g0 * f[0] + g1 * f[1] + g2 * f[2];
                const float dxi = g0 * df[0] + g1 * df[1] + g2 * df[2];
                d += barrier_delta(xi, a * dxi, md.bar_mu, md.bar_delta);
            }
        }
    return d;
}

// grad l_k(z)^T dz
template <int NX>
__device__ float srbd_stage_dphi(const pdilqr_srbd_model& md, const float* x, const float* u,
                                 const float* dx, const float* du, const uint8_t* ct,
                                 const float* xr, const float* ur, bool terminal)
{
    constexpr int NR = NX / 12;
    const float* Wx = terminal ? md.WN : md.W;
    float d = 0.f;
    for (int i = 0; i < NX; ++i) d += Wx[i % 12] * (x[i] - xr[i]) * dx[i];
    if (NR > 1)
        for (int b = 0; b < NR; ++b)
            for (int r = 0; r < 3; ++r) {
                const int n2 = 12 * ((b + 1) % NR) + r;
                d += md.w_form * (x[12 * b + r] - x[n2] - md.d_form[b][r]) * (dx[12 * b + r] - dx[n2]);
            }
    if (terminal) return d;
    for (int i = 0; i < NX; ++i) d += md.Wu[i % 12] * (u[i] - ur[i]) * du[i];
    for (int b = 0; b < NR; ++b)
        for (int j = 0; j < 4; ++j) {
            if (!ct[4 * b + j]) continue;
            const float* f = u + 12 * b + 3 * j;
            const float* df = du + 12 * b + 3 * j;
            for (int c = 0; c < 5; ++c) {
                const float g0 = cone_g(c, 0, md.mu_fric), g1 = cone_g(c, 1, md.mu_fric),
                            g2 = cone_g(c, 2, md.mu_fric);
                float v, d1, d2;
                barrier3(g0 * f[0] + g1 * f[1] + g2 * f[2], md.bar_mu, md.bar_delta, v, d1, d2);
                d += d1 * (g0 * df[0] + g1 * df[1] + g2 * df[2]);
            }
        }
    return d;
}

// | x1 - h(x, u) |_2 for one stage at the trial point z + a dz.  The state
// difference is formed before the trial states are rounded:
//   (x1 - x) + a (dx1 - dx) - dt f(x + a dx, u + a du),
// so the defect is not buried under the rounding of O(1) states.
template <int NX>
__device__ float srbd_stage_defect(const pdilqr_srbd_model& md, const float* x, const float* u,
                                   const float* x1, const float* dx, const float* du,
                                   const float* dx1, const uint8_t* ct, float a)
{
    constexpr int NR = NX / 12;
    float ss = 0.f;
    for (int b = 0; b < NR; ++b) {
        float xt[12], ut[12], xd[12];
        for (int i = 0; i < 12; ++i) {
            xt[i] = x[12 * b + i] + a * dx[12 * b + i];
            ut[i] = u[12 * b + i] + a * du[12 * b + i];
        }
        srbd_xdot(md, xt, ut, ct + 4 * b, xd);
        for (int i = 0; i < 12; ++i) {
            const int j = 12 * b + i;
            const float e = (x1[j] - x[j]) + a * (dx1[j] - dx[j]) - md.dt * xd[i];
            ss += e * e;
        }
    }
    return sqrtf(ss);
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_maxf(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Line-search merit of one instance by the warps of a CTA (columns: the
// ten step sizes, then the current point).  out (shared, 24 doubles):
// [0] J(0), [1] theta(0), [2] dphi, [3+t] J(a_t) - J(0), [13+t] theta(a_t),
// [23] |dz|_inf, [25] |x|_inf.  Ends with __syncthreads.
template <int NX, int NU>
__device__ void merit_block(const pdilqr_srbd_model& md, const float* x, const float* u,
                            const float* dx, const float* du, const float* xr, const float* ur,
                            const uint8_t* ct, const float* x0hat, int N, int nrob, double* out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int col = warp; col < 11; col += nw) {
        double aJ = 0.0, aT = 0.0, aD = 0.0;
        float step = 0.f, xmax = 0.f;
        const float a = col < 10 ? ldexpf(1.f, -col) : 0.f;
        for (int k = lane; k <= N; k += 32) {
            const bool term = k == N;
            const float* xk = x + (int64_t)k * NX;
            const float* uk = u + (int64_t)k * NU;
            const float* dxk = dx + (int64_t)k * NX;
            const float* duk = du + (int64_t)k * NU;
            const uint8_t* ck = ct + (int64_t)k * 4 * nrob;
            const float* xrk = xr + (int64_t)k * NX;
            const float* urk = ur + (int64_t)k * NU;
            if (col < 10) {
                aJ += (double)srbd_stage_dcost<NX>(md, xk, uk, dxk, duk, ck, xrk, urk, a, term);
            } else {
                aJ += (double)srbd_stage_cost<NX>(md, xk, uk, ck, xrk, urk, term);
                aD += (double)srbd_stage_dphi<NX>(md, xk, uk, dxk, duk, ck, xrk, urk, term);
                for (int i = 0; i < NX; ++i) {
                    step = fmaxf(step, fabsf(dxk[i]));
                    xmax = fmaxf(xmax, fabsf(xk[i]));
                }
                if (!term)
                    for (int i = 0; i < NU; ++i) step = fmaxf(step, fabsf(duk[i]));
            }
            if (!term)
                aT += (double)srbd_stage_defect<NX>(md, xk, uk, xk + NX, dxk, duk, dxk + NX, ck, a);
            if (k == 0) {
                float ss = 0.f;
                for (int i = 0; i < NX; ++i) {
                    const float e = x0hat[i] - (xk[i] + a * dxk[i]);
                    ss += e * e;
                }
                aT += (double)sqrtf(ss);
            }
        }
        aJ = warp_sum(aJ);
        aT = warp_sum(aT);
        aD = warp_sum(aD);
        step = warp_maxf(step);
        xmax = warp_maxf(xmax);
        if (lane == 0) {
            if (col < 10) {
                out[3 + col] = aJ;
                out[13 + col] = aT;
            } else {
                out[0] = aJ;
                out[1] = aT;
                out[2] = aD;
                out[23] = (double)step;
                out[25] = (double)xmax;
            }
        }
    }
    __syncthreads();
}

// Filter acceptance (Sec. II-E) on cost differences dJ = J(a) - J(0).
__device__ __forceinline__ bool filter_ok(double th0, double dphi, double thmax, double a,
                                          double dJ, double tha, double c_arm)
{
    if (!(isfinite(dJ) && isfinite(tha))) return false;
    if (th0 > thmax) return tha < th0;
    if (dphi < 0.0) return dJ <= c_arm * a * dphi && tha <= thmax;
    return dJ < 0.0 || tha < th0;
}

}  // namespace pdl
