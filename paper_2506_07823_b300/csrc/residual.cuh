// residual.cuh -- FP64 residual of the LQ KKT system and the update of one
// iterative-refinement step.
//
// For z = (dx, du, dlam) the KKT rows (first-order conditions of Eq. (QP)
// with the Lagrangian of Sec. II-B) are
//   init      s - dx_0                                        = 0
//   x_k       Q dx_k + S^T du_k + q_k + A^T dlam_{k+1} - dlam_k = 0   (k < N)
//   u_k       S dx_k + R du_k + r_k + B^T dlam_{k+1}          = 0   (k < N)
//   dyn_k     A dx_k + B du_k + c_k - dx_{k+1}                = 0   (k < N)
//   term      Q_N dx_N + q_N - dlam_N                         = 0
// Every row is evaluated in double precision from the FP32 data.  The rows
// are also the right-hand side of the correction system: K dz = -rows means
// an LQ problem with the same matrices and vectors
//   s' = s - dx_0, q' = row_x (row_term at N), r' = row_u, c' = row_dyn.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kkt_scan.cuh"

namespace pdl {

struct ResidArgs {
    const float *A, *B, *c, *Q, *R, *S, *q, *r, *s;
    const float *dx, *du, *dlam;
    const int32_t* N;
    const int64_t* off;
    const int64_t* stage_inst;   // [total stages] owning instance of each slot, -1 if none
    int64_t total_stages;
    double* norms;               // [count][4]: |res|, |K|, |z|, |rhs| (max-reduced)
    float *rq, *rr, *rc, *rs;    // optional correction right-hand side (null: skip)
};

__device__ __forceinline__ void atomic_max_pos(double* addr, double v)
{
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(addr), __double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One warp per stage slot; lanes own rows.
template <int NX, int NU>
__global__ void __launch_bounds__(256) kkt_residual_kernel(const __grid_constant__ ResidArgs a)
{
    const int64_t gs = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (gs >= a.total_stages) return;
    const int64_t inst = a.stage_inst[gs];
    if (inst < 0) return;  // slot between instances
    const int N = a.N[inst];
    const int k = (int)(gs - a.off[inst]);
    double res = 0.0, kn = 0.0, zn = 0.0, rn = 0.0;
    const float* dx = a.dx + gs * NX;
    const float* dl = a.dlam + gs * NX;
    if (k < N) {
        const float* A = a.A + gs * NX * NX;
        const float* B = a.B + gs * NX * NU;
        const float* Q = a.Q + gs * NX * NX;
        const float* R = a.R + gs * NU * NU;
        const float* S = a.S ? a.S + gs * NU * NX : nullptr;
        const float* du = a.du + gs * NU;
        const float* dx1 = a.dx + (gs + 1) * NX;
        const float* dl1 = a.dlam + (gs + 1) * NX;
        for (int i = lane; i < NX; i += 32) {
            // x-row
            double v = (double)a.q[gs * NX + i] - (double)dl[i], row = 1.0;
            for (int j = 0; j < NX; ++j) {
                v += (double)Q[i * NX + j] * (double)dx[j] + (double)A[j * NX + i] * (double)dl1[j];
                row += fabs((double)Q[i * NX + j]) + fabs((double)A[j * NX + i]);
            }
            if (S)
                for (int j = 0; j < NU; ++j) {
                    v += (double)S[j * NX + i] * (double)du[j];
                    row += fabs((double)S[j * NX + i]);
                }
            res = fmax(res, fabs(v));
            kn = fmax(kn, row);
            rn = fmax(rn, fabs((double)a.q[gs * NX + i]));
            if (a.rq) a.rq[gs * NX + i] = (float)v;
            // dynamics row
            double d = (double)a.c[gs * NX + i] - (double)dx1[i];
            row = 1.0;
            for (int j = 0; j < NX; ++j) {
                d += (double)A[i * NX + j] * (double)dx[j];
                row += fabs((double)A[i * NX + j]);
            }
            for (int j = 0; j < NU; ++j) {
                d += (double)B[i * NU + j] * (double)du[j];
                row += fabs((double)B[i * NU + j]);
            }
            res = fmax(res, fabs(d));
            kn = fmax(kn, row);
            rn = fmax(rn, fabs((double)a.c[gs * NX + i]));
            if (a.rc) a.rc[gs * NX + i] = (float)d;
            zn = fmax(zn, fmax(fabs((double)dx[i]), fabs((double)dl[i])));
        }
        for (int i = lane; i < NU; i += 32) {
            double v = (double)a.r[gs * NU + i], row = 0.0;
            for (int j = 0; j < NX; ++j) {
                v += (double)B[j * NU + i] * (double)dl1[j];
                row += fabs((double)B[j * NU + i]);
                if (S) {
                    v += (double)S[i * NX + j] * (double)dx[j];
                    row += fabs((double)S[i * NX + j]);
                }
            }
            for (int j = 0; j < NU; ++j) {
                v += (double)R[i * NU + j] * (double)du[j];
                row += fabs((double)R[i * NU + j]);
            }
            res = fmax(res, fabs(v));
            kn = fmax(kn, row);
            rn = fmax(rn, fabs((double)a.r[gs * NU + i]));
            if (a.rr) a.rr[gs * NU + i] = (float)v;
            zn = fmax(zn, fabs((double)du[i]));
        }
    } else {
        const float* Q = a.Q + gs * NX * NX;
        for (int i = lane; i < NX; i += 32) {
            double v = (double)a.q[gs * NX + i] - (double)dl[i], row = 1.0;
            for (int j = 0; j < NX; ++j) {
                v += (double)Q[i * NX + j] * (double)dx[j];
                row += fabs((double)Q[i * NX + j]);
            }
            res = fmax(res, fabs(v));
            kn = fmax(kn, row);
            rn = fmax(rn, fabs((double)a.q[gs * NX + i]));
            if (a.rq) a.rq[gs * NX + i] = (float)v;
            zn = fmax(zn, fmax(fabs((double)dx[i]), fabs((double)dl[i])));
        }
        if (a.rr)
            for (int i = lane; i < NU; i += 32) a.rr[gs * NU + i] = 0.f;
        if (a.rc)
            for (int i = lane; i < NX; i += 32) a.rc[gs * NX + i] = 0.f;
    }
    if (k == 0) {
        for (int i = lane; i < NX; i += 32) {
            const double sv = (double)a.s[inst * NX + i];
            const double d = sv - (double)dx[i];
            res = fmax(res, fabs(d));
            kn = fmax(kn, 1.0);
            rn = fmax(rn, fabs(sv));
            if (a.rs) a.rs[inst * NX + i] = (float)d;
        }
    }
    res = warp_max(res);
    kn = warp_max(kn);
    zn = warp_max(zn);
    rn = warp_max(rn);
    if (lane == 0) {
        double* o = a.norms + inst * 4;
        atomic_max_pos(o + 0, res);
        atomic_max_pos(o + 1, kn);
        atomic_max_pos(o + 2, zn);
        atomic_max_pos(o + 3, rn);
    }
}

// z += dz over n elements (one refinement update).
static __global__ void axpy_kernel(float* __restrict__ z, const float* __restrict__ dz, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] += dz[i];
}

}  // namespace pdl
