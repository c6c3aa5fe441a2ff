// sqp.cuh -- the multiple-shooting SQP of Sec. II-B..II-E in one kernel:
// per iteration the SRBD linearisation (on the fly, inside the scan), the LQ
// KKT solve by the parallel scan, the parallel line search over the ten step
// sizes 2^0..2^-9 and the update of Eq. (linear_rollout).  One CTA per
// instance; no host synchronisation between iterations.
#pragma once

#include "kkt_scan.cuh"
#include "srbd.cuh"

namespace pdl {

enum : int32_t { ST_LINESEARCH = PDILQR_E_LINESEARCH };

struct SqpArgs {
    pdilqr_srbd_model md;
    const float* x0hat;             // [count][n]
    float *x, *u, *lam;             // trajectory (in: warm start, out: solution)
    const float *xref, *uref;
    const uint8_t* contact;
    KktArgs ka;                     // step buffers, policy workspace, batch tables
    int max_iters;
    float tol_step, tol_theta, c_armijo, theta_frac;
    const float* alpha_replay;      // [count][max_iters] or null
    int32_t *iters, *status;        // [count]
    float* alpha;                   // [count][max_iters] or null
    double *J, *theta;              // [count] or null
    float* lqcache;                 // [slots][StageL::IN] linearised-stage cache or null
    int ipc = 0;                    // instances per CTA of the row-per-lane sequential kernel (0: 2)
};

template <int NX, int NU, int W>
struct SqpSmem {
    using SC = ScanSmem<NX, NU, W>;
    static constexpr int MER = (SC::TOTAL + 1) & ~1;             // 8-byte aligned
    static constexpr int SBUF = MER + 2 * 32;                    // 32 doubles
    static constexpr int CTL = SBUF + round4(NX);
    static constexpr int TOTAL = CTL + 8;
    static constexpr size_t BYTES = sizeof(float) * TOTAL;
    static constexpr size_t EXTRA_BYTES = sizeof(float) * (TOTAL - MER);   // extras only
};

template <int NX, int NU, int W, int UW>
__global__ void __launch_bounds__(W * 32 * UW, MinBlocks<W * UW>::value)
    sqp_kernel(const __grid_constant__ SqpArgs a)
{
    using SM = SqpSmem<NX, NU, W>;
    extern __shared__ __align__(16) float smem_all[];
    // scan work areas in shared memory, or in a per-CTA global slice for
    // states whose areas do not fit (shared memory then holds the extras only)
    float* work = a.ka.gws ? a.ka.gws + (int64_t)blockIdx.x * SM::SC::TOTAL : smem_all;
    float* smem = a.ka.gws ? smem_all - SM::MER : smem_all;
    using TL = UnitTiles<W, UW>;
    using UF = UnitFactor<NU, W, UW>;
    const size_t tbase = a.ka.gws ? SM::EXTRA_BYTES : SM::BYTES;
    float* tiles = TL::fit(tbase) ? smem_all + TL::at(tbase) / sizeof(float) : nullptr;
    const size_t fbase = TL::total(tbase);
    float* factors = (a.ka.gws && UF::fit(fbase)) ? smem_all + UF::at(fbase) / sizeof(float) : nullptr;
    const int inst = a.ka.order ? a.ka.order[blockIdx.x] : blockIdx.x;
    if (inst >= a.ka.count) return;
    // tensor-core products (one-chunk large states): TMEM and barrier for the
    // whole kernel, released on its single exit path below
    TcCtx* tc = nullptr;
    if constexpr (UseTc<NX, NU, W, UW>::value) {
        __shared__ TcCtx tcx;
        if (factors) {
            tc_setup(&tcx, UseTc<NX, NU, W, UW>::cols, (a.ka.dbg & PDILQR_DEBUG_TC_SKIP_ISSUE) != 0);
            tc = &tcx;
        }
    }
    const int N = a.ka.N[inst];
    const int64_t off = a.ka.off[inst];
    const int nrob = a.md.nrob;
    double* mer = reinterpret_cast<double*>(smem + SM::MER);  // [0..25] merit, [24] theta_max
    float* sbuf = smem + SM::SBUF;
    float* alpha_sh = smem + SM::CTL;
    int* ctl = reinterpret_cast<int*>(smem + SM::CTL + 1);    // [0] converged flag

    const SrbdSource src{a.md, a.x, a.u, a.lam, a.xref, a.uref, a.contact, nrob, a.lqcache};
    const float* xh = a.x0hat + (int64_t)inst * NX;
    float* x = a.x + off * NX;
    float* u = a.u + off * NU;
    float* lam = a.lam + off * NX;
    const float* dx = a.ka.dx + off * NX;
    const float* du = a.ka.du + off * NU;
    const float* dl = a.ka.dlam + off * NX;
    const float* xr = a.xref + off * NX;
    const float* ur = a.uref + off * NU;
    const uint8_t* ct = a.contact + off * 4 * nrob;

    int status = ST_OK, iters = 0;
    for (int it = 0; it < a.max_iters; ++it) {
        for (int i = threadIdx.x; i < NX; i += blockDim.x) sbuf[i] = xh[i] - x[i];
        __syncthreads();
        const int st = scan_solve<NX, NU, W, UW>(src, a.ka, N, off, sbuf, work, tiles, factors, tc);
        if (st != ST_OK) {
            status = st;
            break;
        }
        iters = it + 1;
        merit_block<NX, NU>(a.md, x, u, dx, du, xr, ur, ct, xh, N, nrob, mer);
        if (threadIdx.x == 0) {
            const double th0 = mer[1], dphi = mer[2];
            if (it == 0) mer[24] = (double)a.theta_frac * fmax(1.0, th0);
            const double thmax = mer[24];
            float alpha = 0.f;
            double th_new = INFINITY;
            if (a.alpha_replay) {
                alpha = a.alpha_replay[(int64_t)inst * a.max_iters + it];
                for (int t = 0; t < 10; ++t)
                    if (alpha == ldexpf(1.f, -t)) th_new = mer[13 + t];
            } else {
                for (int t = 0; t < 10; ++t) {
                    const double at = ldexp(1.0, -t);
                    if (filter_ok(th0, dphi, thmax, at, mer[3 + t], mer[13 + t], a.c_armijo)) {
                        alpha = (float)at;
                        th_new = mer[13 + t];
                        break;
                    }
                }
            }
            // No step accepted while theta(0) already sits at the rounding floor
            // of the FP32 iterate ((N+1) sqrt(n) u |x|_inf): converged at working
            // precision, not a failure.
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
        // Eq. (linear_rollout): x += a dx, u += a du, lam += a dlam
        for (int64_t e = threadIdx.x; e < (int64_t)(N + 1) * NX; e += blockDim.x) {
            x[e] += alpha * dx[e];
            lam[e] += alpha * dl[e];
        }
        for (int64_t e = threadIdx.x; e < (int64_t)N * NU; e += blockDim.x) u[e] += alpha * du[e];
        __syncthreads();
        if (ctl[0]) break;
    }
    if (a.J || a.theta) {
        // merit at the returned iterate (the step buffers still hold the last
        // direction; only the current-point column is read)
        merit_block<NX, NU>(a.md, x, u, dx, du, xr, ur, ct, xh, N, nrob, mer);
    }
    if (tc) tc_teardown(tc);
    if (threadIdx.x == 0) {
        a.iters[inst] = iters;
        a.status[inst] = status;
        if (a.J) a.J[inst] = mer[0];
        if (a.theta) a.theta[inst] = mer[1];
        if (a.alpha)
            for (int it = iters; it < a.max_iters; ++it) a.alpha[(int64_t)inst * a.max_iters + it] = 0.f;
    }
}

// ------------------------------------------------ standalone linearisation
struct LinArgs {
    pdilqr_srbd_model md;
    const float *x, *u, *lam, *xref, *uref;
    const uint8_t* contact;
    float *A, *B, *c, *Q, *R, *S, *q, *r;
    const int32_t* N;
    const int64_t* off;
    const int64_t* stage_inst;
    int64_t total;
    float* work;    // [blocks][StageL::SIZE] global stage areas, or null (shared memory)
};

// SPB stage slots per block, each linearised by a unit of UW warps into a
// stage area in shared memory, or (work != null: stages larger than shared
// memory) into the block's area of a global workspace; blocks stride over
// the slots.
template <int NX, int NU, int SPB, int UW>
__global__ void __launch_bounds__(SPB * 32 * UW) linearize_kernel(const __grid_constant__ LinArgs a)
{
    using L = StageL<NX, NU>;
    constexpr int NT = 32 * UW;
    extern __shared__ __align__(16) float smem[];
    const int unit = threadIdx.x / NT;
    const Grp<NT> g{(int)(threadIdx.x % NT), 1 + unit};
    float* st = a.work ? a.work + (int64_t)blockIdx.x * L::SIZE : smem + unit * L::SIZE;
    const int nrob = a.md.nrob;
    for (int64_t gs = (int64_t)blockIdx.x * SPB + unit; gs < a.total; gs += (int64_t)gridDim.x * SPB) {
        const int64_t inst = a.stage_inst[gs];
        if (inst < 0) continue;   // slot of no instance (uniform over the unit)
        const int N = a.N[inst];
        const int k = (int)(gs - a.off[inst]);
        const bool term = k == N;
        srbd_linearize_stage<NX, NU, NT>(g, st, a.md, a.x + gs * NX, a.u + gs * NU,
                                         term ? nullptr : a.x + (gs + 1) * NX, a.lam + gs * NX,
                                         term ? nullptr : a.lam + (gs + 1) * NX, a.xref + gs * NX,
                                         a.uref + gs * NU, a.contact + gs * 4 * nrob, term);
        for (int e = g.t; e < NX * NX; e += NT) {
            a.Q[gs * NX * NX + e] = st[L::Q + e];
            a.A[gs * NX * NX + e] = term ? 0.f : st[L::A + e];
        }
        for (int e = g.t; e < NX * NU; e += NT) {
            a.B[gs * NX * NU + e] = term ? 0.f : st[L::B + e];
            if (a.S) a.S[gs * NX * NU + e] = 0.f;
        }
        for (int e = g.t; e < NU * NU; e += NT) a.R[gs * NU * NU + e] = term ? 0.f : st[L::R + e];
        for (int i = g.t; i < NX; i += NT) {
            a.q[gs * NX + i] = st[L::q + i];
            a.c[gs * NX + i] = term ? 0.f : st[L::c + i];
        }
        for (int i = g.t; i < NU; i += NT) a.r[gs * NU + i] = term ? 0.f : st[L::r + i];
        g.sync();   // the stage area is rewritten by the next slot
    }
}

// ------------------------------------------------------ standalone merit
struct MeritArgs {
    pdilqr_srbd_model md;
    const float *x, *u, *xref, *uref, *x0hat, *dx, *du;
    const uint8_t* contact;
    const int32_t* N;
    const int64_t* off;
    double* out;   // [count][24]
    int count;
};

template <int NX, int NU>
__global__ void __launch_bounds__(256) merit_kernel(const __grid_constant__ MeritArgs a)
{
    __shared__ double mer[32];
    const int inst = blockIdx.x;
    if (inst >= a.count) return;
    const int N = a.N[inst];
    const int64_t off = a.off[inst];
    const int nrob = a.md.nrob;
    if (threadIdx.x < 32) mer[threadIdx.x] = 0.0;
    __syncthreads();
    merit_block<NX, NU>(a.md, a.x + off * NX, a.u + off * NU, a.dx + off * NX, a.du + off * NU,
                        a.xref + off * NX, a.uref + off * NU, a.contact + off * 4 * nrob,
                        a.x0hat + (int64_t)inst * NX, N, nrob, mer);
    if (threadIdx.x < 24) a.out[(int64_t)inst * 24 + threadIdx.x] = mer[threadIdx.x];
}
// ---------------------------------------- SQP step of the split-scan solve
// The unfused SQP iteration of plans whose scan runs over several CTAs (one
// CTA cannot hold the whole iteration): the stages are linearised into the
// plan's LQ arrays, the split scan solves the KKT system, and this kernel (one
// CTA per instance) evaluates the merit of the ten step sizes, takes the
// filter decision of Sec. II-E with the rules of the fused kernel, applies
// Eq. (linear_rollout) and writes dx_0 of the next KKT solve.  it = -1
// initialises the per-instance state; an instance that has stopped (status,
// convergence or the last iteration) is skipped by later iterations.
struct SqpStepArgs {
    pdilqr_srbd_model md;
    const float* x0hat;
    float *x, *u, *lam;
    const float *xref, *uref;
    const uint8_t* contact;
    const float *dx, *du, *dlam;
    const int32_t* N;
    const int64_t* off;
    int count;
    int it, max_iters;
    float tol_step, tol_theta, c_armijo, theta_frac;
    const float* alpha_replay;     // [count][max_iters] or null
    int32_t *iters, *status;       // [count]
    float* alpha;                  // [count][max_iters] or null
    double *J, *theta;             // [count] or null
    const int32_t* kst;            // [count] status of this iteration's KKT solve
    double* thmax;                 // [count] theta_max, fixed at the first iteration
    int32_t* done;                 // [count] 1: stopped
    float* s;                      // [count][n] dx_0 = xhat_0 - x_0 of the next solve
};

template <int NX, int NU>
__global__ void __launch_bounds__(256) sqp_step_kernel(const __grid_constant__ SqpStepArgs a)
{
    __shared__ double mer[32];
    __shared__ float alpha_sh;
    __shared__ int conv_sh;
    const int inst = blockIdx.x;
    if (inst >= a.count) return;
    const int N = a.N[inst];
    const int64_t off = a.off[inst];
    const int nrob = a.md.nrob;
    const float* xh = a.x0hat + (int64_t)inst * NX;
    float* x = a.x + off * NX;
    float* u = a.u + off * NU;
    float* lam = a.lam + off * NX;
    const float* dx = a.dx + off * NX;
    const float* du = a.du + off * NU;
    const float* dl = a.dlam + off * NX;
    const float* xr = a.xref + off * NX;
    const float* ur = a.uref + off * NU;
    const uint8_t* ct = a.contact + off * 4 * nrob;
    if (a.it < 0) {
        if (threadIdx.x == 0) {
            a.done[inst] = 0;
            a.status[inst] = ST_OK;
            a.iters[inst] = 0;
            if (a.alpha)
                for (int t = 0; t < a.max_iters; ++t) a.alpha[(int64_t)inst * a.max_iters + t] = 0.f;
        }
        for (int i = threadIdx.x; i < NX; i += blockDim.x) a.s[(int64_t)inst * NX + i] = xh[i] - x[i];
        return;
    }
    if (a.done[inst]) return;   // uniform over the CTA
    const int it = a.it;
    int status = a.kst[inst];
    bool stop = status != ST_OK;
    if (!stop) {
        if (threadIdx.x < 32) mer[threadIdx.x] = 0.0;
        __syncthreads();
        merit_block<NX, NU>(a.md, x, u, dx, du, xr, ur, ct, xh, N, nrob, mer);
        if (threadIdx.x == 0) {
            const double th0 = mer[1], dphi = mer[2];
            if (it == 0) a.thmax[inst] = (double)a.theta_frac * fmax(1.0, th0);
            const double thmax = a.thmax[inst];
            float alpha = 0.f;
            double th_new = INFINITY;
            if (a.alpha_replay) {
                alpha = a.alpha_replay[(int64_t)inst * a.max_iters + it];
                for (int t = 0; t < 10; ++t)
                    if (alpha == ldexpf(1.f, -t)) th_new = mer[13 + t];
            } else {
                for (int t = 0; t < 10; ++t) {
                    const double at = ldexp(1.0, -t);
                    if (filter_ok(th0, dphi, thmax, at, mer[3 + t], mer[13 + t], a.c_armijo)) {
                        alpha = (float)at;
                        th_new = mer[13 + t];
                        break;
                    }
                }
            }
            // converged at the rounding floor of the FP32 iterate (as the fused kernel)
            const double floor_th = (double)(N + 1) * sqrt((double)NX) * 0x1p-23 * fmax(1.0, mer[25]);
            const bool at_floor = alpha == 0.f && th0 <= floor_th && !a.alpha_replay;
            alpha_sh = at_floor ? -1.f : alpha;
            conv_sh = (at_floor || (mer[23] < (double)a.tol_step && th_new < (double)a.tol_theta)) ? 1 : 0;
            if (a.alpha) a.alpha[(int64_t)inst * a.max_iters + it] = alpha;
            a.iters[inst] = it + 1;
        }
        __syncthreads();
        const float alpha = alpha_sh;
        if (alpha == 0.f) {
            status = ST_LINESEARCH;
            stop = true;
        } else if (alpha < 0.f) {
            stop = true;
        } else {
            for (int64_t e = threadIdx.x; e < (int64_t)(N + 1) * NX; e += blockDim.x) {
                x[e] += alpha * dx[e];
                lam[e] += alpha * dl[e];
            }
            for (int64_t e = threadIdx.x; e < (int64_t)N * NU; e += blockDim.x) u[e] += alpha * du[e];
            __syncthreads();
            stop = conv_sh != 0;
        }
    }
    if (it + 1 >= a.max_iters) stop = true;
    if (stop) {
        if (a.J || a.theta) {
            // merit at the returned iterate (only the current-point column is read)
            __syncthreads();
            if (threadIdx.x < 32) mer[threadIdx.x] = 0.0;
            __syncthreads();
            merit_block<NX, NU>(a.md, x, u, dx, du, xr, ur, ct, xh, N, nrob, mer);
        }
        if (threadIdx.x == 0) {
            a.status[inst] = status;
            a.done[inst] = 1;
            if (a.J) a.J[inst] = mer[0];
            if (a.theta) a.theta[inst] = mer[1];
        }
    } else {
        for (int i = threadIdx.x; i < NX; i += blockDim.x) a.s[(int64_t)inst * NX + i] = xh[i] - x[i];
    }
}


}  // namespace pdl
